// pass_kernels.cuh - line-pass kernels of the TSSP step (included by the
// per-precision translation units pass_f32.cu / pass_f64.cu).
//
// One launch sweeps every line of one axis of every instance once: load the
// line's points into registers, run up to three pointwise substeps and two
// transforms along that axis, optionally reduce, and store.  The real-time
// step of the paper's TSSP scheme is a product of such sweeps (x rows carry
// the nonlinear substep, the last-transformed axis carries the kinetic one).
#pragma once
#include <mutex>

#include "fft_tile.cuh"
#include "gpe_internal.h"

namespace gpe {

__device__ __forceinline__ void sincos_r(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

// exp(-i th) - 1 = (cos th - 1, -sin th).  Double precision: from the half
// angle, (-2 sin^2(th/2), -sin th).  Single precision, |th| <= 1/2: the
// Maclaurin series of cos th - 1 and sin th to the th^10 / th^11 terms
// (truncation below 1e-11 relative), evaluated by Horner's rule in th^2;
// larger angles fall back to sincosf of the half angle.
__device__ __forceinline__ double2 phase_offset(double th)
{
    double s, c;
    sincos(0.5 * th, &s, &c);
    return mk(-2.0 * s * s, -2.0 * s * c);
}
// short forms for |th| <= 1/16 (Maclaurin series of cos th - 1 and sin th).
// double: terms to th^12 / th^13, truncation below 1e-27;
// float: terms to th^6 / th^5, truncation below 1e-12 (sin) and 1e-14 (cos),
// so the modulus of 1 + w stays one to about 1e-13
__device__ __forceinline__ double2 phase_offset_small(double th)
{
    const double u = th * th;
    const double cm =
        u * fma(u, fma(u, fma(u, fma(u, fma(u, 1.0 / 479001600.0, -1.0 / 3628800.0), 1.0 / 40320.0), -1.0 / 720.0),
                       1.0 / 24.0),
                -0.5);
    const double sn =
        th * fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, 1.0 / 6227020800.0, -1.0 / 39916800.0), 1.0 / 362880.0),
                                         -1.0 / 5040.0),
                                 1.0 / 120.0),
                         -1.0 / 6.0),
                 1.0);
    return mk(cm, -sn);
}
__device__ __forceinline__ float2 phase_offset_small(float th)
{
    const float u = th * th;
    const float cm = u * fmaf(u, fmaf(u, -1.38888889e-3f, 4.16666667e-2f), -0.5f);
    const float sn = th * fmaf(u, fmaf(u, 8.33333333e-3f, -1.66666667e-1f), 1.0f);
    return mk(cm, -sn);
}
__device__ __forceinline__ float2 phase_offset(float th)
{
    if (fabsf(th) <= 0.5f) {
        const float u = th * th;
        const float cm = u * fmaf(u, fmaf(u, fmaf(u, fmaf(u, -2.75573192e-7f, 2.48015873e-5f), -1.38888889e-3f),
                                           4.16666667e-2f), -0.5f);
        const float sn = th * fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, -2.50521084e-8f, 2.75573192e-6f),
                                                          -1.98412698e-4f), 8.33333333e-3f), -1.66666667e-1f), 1.0f);
        return mk(cm, -sn);
    }
    float s, c;
    sincosf(0.5f * th, &s, &c);
    return mk(-2.0f * s * s, -2.0f * s * c);
}

// v_e <- v_e (1 + w_e), w_e = exp(-i th_e) - 1, for the E angles a thread
// holds: the short series for every angle of at most 1/16 (the usual case:
// dt |V + g|psi|^2| is far below it), the long form for the others.  The
// choice is made per element, so a point's result does not depend on which
// lines share its warp (tile shapes and kernels with other thread layouts
// give the same bits); a warp whose angles are all small takes one branch.
template <typename C, typename R, int E>
__device__ __forceinline__ void apply_phase(C (&v)[E], const R (&th)[E])
{
#pragma unroll
    for (int e = 0; e < E; ++e) {
        auto w = phase_offset_small(th[e]);
        if (fabs(th[e]) > (R)0.0625) w = phase_offset(th[e]);
        v[e] = cmadd1(v[e], w);
    }
}

// Tile shapes.  Each pass kind has two compiled shapes, VAR 0 (the default)
// and VAR 1; the plan autotuner times both on the plan's grid and keeps the
// faster (the arithmetic per line is the same in both, so results are too).
//
// Strided lines (y, z).  complex64 VAR 0: tiles of at most 8192 points and 16
// adjacent lines, so every point row of a tile is a 128-byte segment (one CTA
// of <= 1024 threads per SM); with 8 lines (64-byte pieces) the z sweep of a
// 512^3 grid, whose consecutive points are 2 MiB apart, ran at under half the
// copy bandwidth.  VAR 1: 4096 points / 8 lines, two CTAs per SM.
// complex128 VAR 0: 2048 points / 4 lines (64-byte pieces), two CTAs per SM;
// VAR 1: 4096 points / 8 lines.
// Contiguous rows (x).  A split tile holds a fraction of the points and lines
// with the swizzled shared layout and several CTAs per SM: each lane's points
// lie in its own row, and fewer rows per warp request with longer pieces of
// each measured faster for complex64 rows of up to 512 points.  Rows of 256
// or 512 points: tiles of 512 points (shape 0: 1 row of 512 or 2 of 256, each
// warp request reading 256 or 128 contiguous bytes of a row) or 4 rows
// (shape 1) - 512^3 x pass with 4 / 2 / 1 rows: 0.839 / 0.716 / 0.705 ms
// (fixed-program kernels; 4 rows beat 8 in earlier builds, 1.27 -> 1.07 ms).  Shorter complex64 rows (tiny CTAs otherwise): 4 rows (shape 0)
// or the unsplit tile (shape 1).  Longer or complex128 rows: shape 0 is the
// unsplit tile, shape 1 the half tile.
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr bool rows_split()
{
    constexpr bool short_c64 = sizeof(R) == 4 && N <= 512;
    return ROWS && N >= 8 && (short_c64 ? (N >= 256 || VAR == 0) : VAR == 1);
}
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr int pick_lines()
{
    constexpr bool c64 = sizeof(R) == 4;
    int maxpts = c64 ? 4096 : 2048, lmax = c64 ? 8 : 4;
    if (ROWS) {
        if (rows_split<R, N, ROWS, VAR>()) {
            // complex64 rows of 256 or 512 points: tiles of 512 points (shape 0:
            // 2 rows of 256, 1 row of 512) or 4 rows (shape 1)
            const bool small = c64 && N >= 256 && N <= 512 && VAR == 0;
            maxpts /= small ? 8 : 2;
            lmax /= small ? 4 : 2;
        }
    } else if (c64 ? VAR == 0 : VAR == 1) {
        maxpts *= 2;
        lmax *= 2;
    }
    int L = maxpts / N;
    if (L > lmax) L = lmax;
    if (L < 1) L = 1;
    return L;
}
// the on-chip 1D kernel keeps whole lines per thread group (row layout)
template <typename R, int N> __host__ __device__ constexpr int pick_lines_1d()
{
    constexpr int maxpts = sizeof(R) == 4 ? 8192 : 4096;
    int L = maxpts / N;
    if (L > 16) L = 16;
    if (L < 1) L = 1;
    return L;
}

// Sum one double per thread over the TPL threads of each line in a fixed
// tree order; every thread of the line receives the line's total.
template <int L, int TPL>
__device__ __forceinline__ double line_sum(double x, double *red, int l, int tl)
{
    red[tl * L + l] = x;
    __syncthreads();
#pragma unroll 1
    for (int s = TPL / 2; s > 0; s >>= 1) {
        if (tl < s) red[tl * L + l] += red[(tl + s) * L + l];
        __syncthreads();
    }
    double r = red[l];
    __syncthreads();
    return r;
}

// Offset of a product of two unit factors held as offsets a, b from one:
// (1 + a)(1 + b) - 1 = a + b + ab, summed with error-free transformations
// (two-sum, two-product) and returned as a hi + lo float pair, so that the
// product is applied in offset form (v + v c, see uomul) with one rounding.
// The unit-factor form (umul) of the same product would be biased for small
// angles: its real part rounds to exactly one, and the inner fused product
// v.y * 1 + (tiny) then rounds the second-order term away every time (a
// norm gain of about angle^2 / 2 per application).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float4 offset_product(float4 a, float4 b)
{
    // ab: exact products of the hi parts, the cross terms with the lo parts
    // in plain arithmetic (of order 1e-8 |ab|)
    const float p1 = a.x * b.x, e1 = fmaf(a.x, b.x, -p1);
    const float p2 = a.y * b.y, e2 = fmaf(a.y, b.y, -p2);
    const float p3 = a.x * b.y, e3 = fmaf(a.x, b.y, -p3);
    const float p4 = a.y * b.x, e4 = fmaf(a.y, b.x, -p4);
    const float xl = (e1 - e2) + ((a.x * b.z + a.z * b.x) - (a.y * b.w + a.w * b.y));
    const float yl = (e3 + e4) + ((a.x * b.w + a.z * b.y) + (a.y * b.z + a.w * b.x));
    float sx, ex, t, tx, ux, vx;
    two_sum(p1, -p2, sx, ex);
    two_sum(a.x, b.x, t, tx);
    two_sum(t, sx, ux, vx);
    const float lx = vx + (tx + (ex + (xl + (a.z + b.z))));
    float sy, ey, ty, uy, vy;
    two_sum(p3, p4, sy, ey);
    two_sum(a.y, b.y, t, ty);
    two_sum(t, sy, uy, vy);
    const float ly = vy + (ty + (ey + (yl + (a.w + b.w))));
    float hx, gx, hy, gy;
    two_sum(ux, lx, hx, gx);
    two_sum(uy, ly, hy, gy);
    return make_float4(hx, hy, gx, gy);
}
__device__ __forceinline__ double2 offset_product(double2 a, double2 b)
{
    return make_double2(a.x + b.x + (a.x * b.x - a.y * b.y), a.y + b.y + (a.x * b.y + a.y * b.x));
}

// pointwise substep on the E points (indices tl + TPL*e on this axis) of one line
// inst: position of the instance in this launch (renormalisation factor);
// ti: its parameter/table slot
// off: offset of the line's first point within its instance (sampled potential)
template <typename R, int E, int TPL>
__device__ __forceinline__ void point_op(int op, typename CT<R>::C (&v)[E], const PassArgs &a, int inst,
                                         int ti, int c0, int c1, int tl, int64_t off)
{
    using C = typename CT<R>::C;
    if (op == OP_NONE) return;
    using U = typename UT<R>::U;
    if (op == OP_KREAL) {
        // tables hold exp(-i k_a^2 dt/2) - 1; the 1/N of the inverse transform is exact
        const U *kt = static_cast<const U *>(a.kt_ax);
        const R invn = (R)a.inv_n;
        const U *k0 = static_cast<const U *>(a.kt_o0);
        const U *k1 = static_cast<const U *>(a.kt_o1);
        if (!k0 && !k1) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cscale(uomul(v[e], kt[tl + TPL * e]), invn);
            return;
        }
        // the factors of the line's other axes, combined once per line into
        // one offset to twice the working precision
        U fl = offset_product(k0 ? k0[c0] : U{}, k1 ? k1[c1] : U{});
        if constexpr (sizeof(R) == 4) {
            if (a.dither)
                fl = offset_product(fl, make_float4((float)a.dk[0], (float)a.dk[1], (float)a.dk[2], (float)a.dk[3]));
        }
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(uomul(uomul(v[e], kt[tl + TPL * e]), fl), invn);
        return;
    }
    if (op == OP_KIMAG) {
        R fl = (R)1;
        if (a.ki_o0) fl *= static_cast<const R *>(a.ki_o0)[c0];
        if (a.ki_o1) fl *= static_cast<const R *>(a.ki_o1)[c1];
        const R *ki = static_cast<const R *>(a.ki_ax);
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(v[e], fl * ki[tl + TPL * e]);
        return;
    }
    if (op == OP_SCALE || op == OP_SCALE_NIMAG) {
        const R s = (R)a.scale[inst];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(v[e], s);
        if (op == OP_SCALE) return;
    }
    const R gc = (R)(a.g[ti] * a.nl_c);
    if (op == OP_NREAL) {
        // trap tables hold exp(-i V_a c) - 1
        const U *vax = static_cast<const U *>(a.vt_ax);
        const U *v0 = static_cast<const U *>(a.vt_o0);
        const U *v1 = static_cast<const U *>(a.vt_o1);
        const U f0 = v0 ? v0[(int64_t)ti * a.o0n + c0] : U{};
        const U f1 = v1 ? v1[(int64_t)ti * a.o1n + c1] : U{};
        // separate paths with and without a sampled potential keep the
        // common one free of its address arithmetic (fewer live registers)
        R th[E];
        const R dphi = (R)a.dphi;      // undoes the kinetic substep's dither (0 when off)
        if (a.vsamp) {
            const R *vs = static_cast<const R *>(a.vsamp) + off;
            const R cc = (R)a.nl_c;
#pragma unroll
            for (int e = 0; e < E; ++e)
                th[e] = fma(vs[(int64_t)(tl + TPL * e) * a.estride], cc, gc * cabs2(v[e])) - dphi;
            apply_phase<C, R, E>(v, th);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) th[e] = gc * cabs2(v[e]) - dphi;
            apply_phase<C, R, E>(v, th);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C x = v[e];
            if (vax) x = uomul(x, vax[(int64_t)ti * a.nax + tl + TPL * e]);
            if (v0) x = uomul(x, f0);
            if (v1) x = uomul(x, f1);
            v[e] = x;
        }
        return;
    }
    // OP_NIMAG / OP_SCALE_NIMAG
    const R *iax = static_cast<const R *>(a.vi_ax);
    R fl = (R)1;
    if (a.vi_o0) fl *= static_cast<const R *>(a.vi_o0)[(int64_t)ti * a.o0n + c0];
    if (a.vi_o1) fl *= static_cast<const R *>(a.vi_o1)[(int64_t)ti * a.o1n + c1];
    const R *vs = static_cast<const R *>(a.vsamp);
    const R cc = (R)a.nl_c;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        R th = gc * cabs2(v[e]);
        if (vs) th = fma(vs[off + (int64_t)(tl + TPL * e) * a.estride], cc, th);
        R f = fl * exp_r(-th);
        if (iax) f *= iax[(int64_t)ti * a.nax + tl + TPL * e];
        v[e] = cscale(v[e], f);
    }
}

// asynchronous global -> shared copies of one point (cp.async, no register staging)
__device__ __forceinline__ void cp_async_point(void *smem, const float2 *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g));
}
__device__ __forceinline__ void cp_async_point(void *smem, const double2 *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

// ---- tensor-memory-accelerator tile copies with an mbarrier per buffer
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// order this CTA's earlier ordinary shared-memory accesses before later copies into it
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// wait for the given phase parity of a barrier, for at most ~2 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
template <int K> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

// Geometry of the line a thread works on in a given tile.
struct LineGeom {
    int64_t lg, li, off;   // off: offset of the line start from the instance base
    int inst, ti, c0, c1;
    bool valid;
};
template <int L>
__device__ __forceinline__ LineGeom line_geom(const PassArgs &a, int64_t tile, int l)
{
    LineGeom g;
    g.lg = a.line0 + tile * L + l;
    g.valid = g.lg < a.lines_total;
    g.inst = g.valid ? int(g.lg >> a.lg_lpi) : 0;
    g.ti = a.slot_of ? a.slot_of[g.inst] : g.inst;
    g.li = g.lg & ((int64_t(1) << a.lg_lpi) - 1);
    g.c0 = int(g.li & (a.o0n - 1));
    g.c1 = int(g.li >> a.lg_o0);
    g.off = (g.li & ((int64_t(1) << a.lg_A) - 1)) + (g.li >> a.lg_A) * a.Sb;
    return g;
}
// base pointers of an instance (inst_ptr indirection or back-to-back storage)
template <typename C>
__device__ __forceinline__ const C *inst_src(const PassArgs &a, int inst)
{
    return a.inst_ptr ? static_cast<const C *>(a.inst_ptr[inst]) : static_cast<const C *>(a.src) + inst * a.inst_stride;
}
template <typename C> __device__ __forceinline__ C *inst_dst(const PassArgs &a, int inst)
{
    return a.inst_ptr ? static_cast<C *>(a.inst_ptr[inst]) : static_cast<C *>(a.dst) + inst * a.inst_stride;
}

// Per-line sums for the LPT lines of every thread: each line's TPL partial
// values are added in a fixed tree order; all threads of the group receive
// the totals.
template <int L, int TPL, int LPT>
__device__ __forceinline__ void group_sum(double (&x)[LPT], double *red, int l0, int tl)
{
#pragma unroll
    for (int ln = 0; ln < LPT; ++ln) red[tl * L + l0 + ln] = x[ln];
    __syncthreads();
#pragma unroll 1
    for (int s = TPL / 2; s > 0; s >>= 1) {
        if (tl < s) {
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) red[tl * L + l0 + ln] += red[(tl + s) * L + l0 + ln];
        }
        __syncthreads();
    }
#pragma unroll
    for (int ln = 0; ln < LPT; ++ln) x[ln] = red[l0 + ln];
    __syncthreads();
}

// The same tree for complex64 passes, on double-float (hi + lo) values held in
// FP32: a double-precision add is one warp instruction per 64 cycles per SM
// sub-partition on this GPU, so per-thread and per-line sums of float
// quantities are accumulated with error-free FP32 transformations (TwoSum)
// instead, to about 2^-44 relative, and converted to double once per line.
__device__ __forceinline__ void df_acc(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}
__device__ __forceinline__ void df_add(float &hi, float &lo, float bh, float bl)
{
    const float s = hi + bh;
    const float bb = s - hi;
    const float t = ((hi - (s - bb)) + (bh - bb)) + (lo + bl);
    hi = s + t;
    lo = t - (hi - s);
}
// The tree adds tl + s into tl for s = TPL/2, ..., 1, like group_sum, so
// every tile shape adds in one order.  Thread t works on line t mod NP at
// position tl = t div NP (NP = L / LPT): a warp holds 32/NP consecutive
// positions of each of its lines, so the levels with s < 32/NP pair lanes of
// one warp (lane xor s*NP) and run as shuffles; only the levels above them go
// through shared memory and barriers.  The result is valid where tl == 0.
template <int L, int TPL, int LPT>
__device__ __forceinline__ void group_sum_df(float (&hi)[LPT], float (&lo)[LPT], float2 *red, int l0, int tl)
{
    constexpr int NP = L / LPT;
    constexpr bool WARP = NP <= 32 && 32 % NP == 0 && (NP * TPL) % 32 == 0;   // whole warps, lines interleaved
    constexpr int SW = WARP ? (32 / NP < TPL ? 32 / NP : TPL) : 1;            // positions of a line per warp
    if constexpr (TPL > SW) {
#pragma unroll
        for (int ln = 0; ln < LPT; ++ln) red[tl * L + l0 + ln] = make_float2(hi[ln], lo[ln]);
        __syncthreads();
#pragma unroll 1
        for (int s = TPL / 2; s >= SW; s >>= 1) {
            if (tl < s) {
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) {
                    float2 u = red[tl * L + l0 + ln];
                    const float2 w = red[(tl + s) * L + l0 + ln];
                    df_add(u.x, u.y, w.x, w.y);
                    red[tl * L + l0 + ln] = u;
                }
            }
            __syncthreads();
        }
        if (tl < SW) {
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) {
                const float2 u = red[tl * L + l0 + ln];
                hi[ln] = u.x;
                lo[ln] = u.y;
            }
        }
        __syncthreads();     // the next reduction reuses red
    }
#pragma unroll
    for (int s = SW / 2; s >= 1; s >>= 1) {
#pragma unroll
        for (int ln = 0; ln < LPT; ++ln) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi[ln], s * NP);
            const float ol = __shfl_xor_sync(0xffffffffu, lo[ln], s * NP);
            df_add(hi[ln], lo[ln], oh, ol);
        }
    }
}

// lines carried by each thread.  Two lines per thread (16-byte shared accesses,
// one twiddle read for both) measured slower on the strided axes at 512^3
// (occupancy halves at 122 registers), so each thread carries one line.
template <typename R> __host__ __device__ constexpr int lines_per_thread() { return 1; }

// One sweep over every line of one axis.  Threads are laid out across the
// lines of a tile (a thread carries LPT adjacent lines at points t / NP +
// TPL*e), so that warp-wide accesses to consecutive lines are contiguous for
// the y and z axes and every twiddle read in a Stockham pass is a broadcast
// shared by the thread's lines.  Tiles are software-pipelined: the points of
// tile i+2 are copied into one of two shared buffers with cp.async while tile
// i is transformed in the other.
// points per thread: 16 for strided complex64 lines of at least 16 points (two
// butterflies per thread and pass: the 512^3 y sweep 0.51 -> 0.45 ms, z 0.92 ->
// 0.90 ms), else 8; rows keep 8 (16 measured slower there).  Every tile shape
// of a pass kind uses the same count, so the per-line reductions add in the
// same order whichever shape the tuner picks.
template <typename R, int N, bool ROWS> __host__ __device__ constexpr int pass_points_per_thread()
{
    return (!ROWS && sizeof(R) == 4 && N >= 256 && N <= 1024) ? 32
           : (!ROWS && sizeof(R) == 4 && N >= 16)              ? 16
                                                               : Radix<N>::E;
}

// Shared layout of the transform exchanges: rows of the split tiles are
// swizzled (see rows_split), strided tiles are not.  (Swizzling the 8-line
// strided tiles of 32 points per thread removes the 4-way bank conflicts of
// their first exchange, but with it the 512^3 y sweep ran at 0.475 ms
// against 0.347 ms without.)  A tile staged by the copy engine is read
// with the plain index.
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr bool pass_swizzle()
{
    return rows_split<R, N, ROWS, VAR>();
}
// Strided tiles of 32 points per thread whose point rows are narrower than a
// bank row take the padded exchange layout instead (no index arithmetic
// added; see GTile).
template <typename R, int N, bool ROWS> __host__ __device__ constexpr bool pass_pad()
{
    return !ROWS && pass_points_per_thread<R, N, ROWS>() == 32;
}
template <typename R, int N, bool ROWS, int VAR>
using PassTile = GTile<R, N, pick_lines<R, N, ROWS, VAR>(), lines_per_thread<R>(), pass_swizzle<R, N, ROWS, VAR>(),
                       pass_points_per_thread<R, N, ROWS>(), pass_pad<R, N, ROWS>()>;

// dynamic shared memory of one CTA without the transform scratch: two staging
// buffers, per-line reduction scratch, twiddles, two mbarriers
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr size_t pass_smem_base()
{
    using T = PassTile<R, N, ROWS, VAR>;
    return 2 * sizeof(typename T::C) * T::BUF_POINTS + sizeof(double) * (size_t)(T::SMEM_POINTS / T::E) +
           sizeof(typename T::U) * N + 2 * sizeof(uint64_t);
}
// CTAs per SM the registers are budgeted for: 4 per SM for split rows (1024 /
// threads per CTA, at most 16), else 2 (1 for CTAs of more than 512 threads),
// never more than fit in the SM's shared memory
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr int pass_min_blocks()
{
    constexpr int nt = PassTile<R, N, ROWS, VAR>::NT;
    constexpr int want = 1024 / nt > 16 ? 16 : 1024 / nt;
    // (strided tiles of 32 points per thread keep 2: capping their registers
    // for a third CTA, 170, made the 512^3 y sweep slower, 0.347 -> 0.475 ms)
    constexpr int b = rows_split<R, N, ROWS, VAR>() && want > 2 ? want : (nt > 512 ? 1 : 2);
    constexpr int fit = (int)(227 * 1024 / (pass_smem_base<R, N, ROWS, VAR>() + 1024));
    return b < fit ? b : (fit > 0 ? fit : 1);
}
// A third tile-sized region lets the transform passes alternate between two
// regions (one barrier per pass instead of two).  It is added to kernels built
// for one CTA per SM, whose shared memory is otherwise partly idle, where it
// fits: 512^3 complex64 z sweep 0.810 -> 0.797 ms; with two CTAs per SM the y
// sweep slowed (0.411 -> 0.433 ms).
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr bool pass_ping()
{
    using T = PassTile<R, N, ROWS, VAR>;
    constexpr size_t with = pass_smem_base<R, N, ROWS, VAR>() + sizeof(typename T::C) * T::BUF_POINTS;
    return T::PL::P > 1 && pass_min_blocks<R, N, ROWS, VAR>() == 1 && with + 1024 <= 227 * 1024;
}
template <typename R, int N, bool ROWS, int VAR> __host__ __device__ constexpr size_t pass_smem_bytes()
{
    using T = PassTile<R, N, ROWS, VAR>;
    return pass_smem_base<R, N, ROWS, VAR>() +
           (pass_ping<R, N, ROWS, VAR>() ? sizeof(typename T::C) * T::BUF_POINTS : 0);
}

// Sweep programs compiled with their slots fixed: the passes of the real- and
// imaginary-time steps, with the first and last x sweeps of a real-time call.
// Program 0 reads the slots from the arguments (every other sweep:
// diagnostics, spectra, the final renormalisation).  The real-time programs
// give the generic kernel's bits (tested); the imaginary-time ones (5-7) can
// round differently from it in the last place (seen on the decay sweeps, cause
// not identified), well inside the parity tolerances.
struct SweepProg {
    int op_pre, fft1, op_mid, fft2, op_post, red;
};
__host__ __device__ constexpr SweepProg sweep_prog(int p)
{
    return p == 1   ? SweepProg{OP_NONE, -1, OP_KREAL, 1, OP_NONE, RED_NONE}    // F, kinetic, I
           : p == 2 ? SweepProg{OP_NONE, 1, OP_NONE, 0, OP_NONE, RED_NONE}      // I
           : p == 3 ? SweepProg{OP_NONE, -1, OP_NONE, 0, OP_NONE, RED_NONE}     // F
           : p == 4 ? SweepProg{OP_NONE, 1, OP_NREAL, -1, OP_NONE, RED_NONE}    // I, nonlinear, F
           : p == 5 ? SweepProg{OP_SCALE_NIMAG, -1, OP_NONE, 0, OP_NONE, RED_NONE}   // scale, decay, F
           : p == 6 ? SweepProg{OP_NONE, -1, OP_KIMAG, 1, OP_NONE, RED_NONE}    // F, kinetic decay, I
           : p == 7 ? SweepProg{OP_NONE, 1, OP_NIMAG, 0, OP_NONE, RED_NORM}     // I, decay, norm
           : p == 8 ? SweepProg{OP_NREAL, -1, OP_NONE, 0, OP_NONE, RED_NONE}    // first half-step, F
           : p == 9 ? SweepProg{OP_NONE, 1, OP_NREAL, 0, OP_NONE, RED_NONE}     // I, last half-step
                    : SweepProg{-1, -1, -1, -1, -1, -1};
}
constexpr int NUM_SWEEP_PROGS = 9;
inline int sweep_prog_of(const PassArgs &a)
{
    if (a.generic) return 0;
    for (int p = 1; p <= NUM_SWEEP_PROGS; ++p) {
        const SweepProg q = sweep_prog(p);
        if (a.op_pre == q.op_pre && a.fft1 == q.fft1 && a.op_mid == q.op_mid && a.fft2 == q.fft2 &&
            a.op_post == q.op_post && a.red == q.red)
            return p;
    }
    return 0;
}

template <typename R, int N, bool ROWS, int VAR, int PROG>
__global__ void __launch_bounds__(PassTile<R, N, ROWS, VAR>::NT, (pass_min_blocks<R, N, ROWS, VAR>()))
    k_pass(const PassArgs a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr SweepProg PP = sweep_prog(PROG);
    const int op_pre = PROG ? PP.op_pre : a.op_pre, op_mid = PROG ? PP.op_mid : a.op_mid;
    const int op_post = PROG ? PP.op_post : a.op_post, rmode = PROG ? PP.red : a.red;
    const int fft1 = PROG ? PP.fft1 : a.fft1, fft2 = PROG ? PP.fft2 : a.fft2;
    constexpr int LPT = lines_per_thread<R>();
    constexpr int L = pick_lines<R, N, ROWS, VAR>();
    using T = PassTile<R, N, ROWS, VAR>;
    using C = typename T::C;
    using U = typename T::U;
    constexpr int E = T::E, TPL = T::TPL;
    constexpr bool PING = pass_ping<R, N, ROWS, VAR>();
    extern __shared__ __align__(128) unsigned char smraw[];
    C *buf0 = reinterpret_cast<C *>(smraw);
    C *buf1 = buf0 + T::BUF_POINTS;
    constexpr size_t tiles_bytes = (PING ? 3 : 2) * sizeof(C) * T::BUF_POINTS;
    C *const scr = PING ? buf1 + T::BUF_POINTS : nullptr;
    double *red = reinterpret_cast<double *>(smraw + tiles_bytes);
    U *tw = reinterpret_cast<U *>(smraw + tiles_bytes + sizeof(double) * N * L / E);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smraw + tiles_bytes + sizeof(double) * N * L / E + sizeof(U) * N);
    const int t = threadIdx.x, l0 = (t % T::NP) * LPT, tl = t / T::NP;
    T::load_twiddles(tw, static_cast<const U *>(a.tw), t, T::NT);

    // Strided tiles (point i of line l at i*L + l, the layout of a box of L
    // lines by tma_box points) can be fetched by the copy engine: thread 0
    // issues the boxes of a tile against the buffer's mbarrier and every
    // thread waits on it.  Other tiles go through per-thread cp.async.
    const bool tma = !ROWS && LPT == 1 && a.tma_chunks > 0;
    if (tma) {
        if (t == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            mbar_init_fence();
        }
        __syncthreads();
    }
    int issued[2] = {0, 0};   // boxes sets issued into each buffer (thread 0)
    // Programmatic dependent launch: everything above (twiddles, barriers)
    // touches nothing the previous kernel of the stream writes, so it may
    // overlap that kernel's tail; the state is read only after this wait,
    // which returns once the previous grid has completed and its writes are
    // visible.  Without the launch attribute it returns at once.
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (a.pdl_early) asm volatile("griddepcontrol.launch_dependents;\n" :::);
    // an imaginary-time run that has met its stopping rule: nothing to do
    // (no copy has been issued yet; every thread reads the same word)
    if (a.stop && *reinterpret_cast<const volatile int *>(a.stop)) return;

    auto stage = [&](int64_t tile, C *buf, int b) {
        if (tma) {
            if (t == 0 && tile < a.ntiles) {
                const int64_t lg = a.line0 + tile * L;
                const int inst = int(lg >> a.lg_lpi);
                const int64_t li = lg & ((int64_t(1) << a.lg_lpi) - 1);
                const int c0 = int(li & (a.o0n - 1)), c1 = int(li >> a.lg_o0);
                const int x = c0 * (int)(sizeof(C) / 8);      // complex128 rows are pairs of doubles
                fence_async_shared();
                mbar_expect_tx(&mbar[b], (unsigned)(sizeof(C) * N * L) + (unsigned)a.tx_extra);
                for (int c = 0; c < a.tma_chunks; ++c) {
                    const int pa = c * a.tma_box;
                    if (a.axis == 1) tma_load_4d(buf + pa * L, &tmap, x, pa, c1, inst, &mbar[b]);
                    else tma_load_4d(buf + pa * L, &tmap, x, c1, pa, inst, &mbar[b]);
                }
                ++issued[b];
            }
            return;
        }
        if (tile < a.ntiles) {
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) {
                const LineGeom g = line_geom<L>(a, tile, l0 + ln);
                if (g.valid) {
                    const C *src = inst_src<C>(a, g.inst) + g.off;
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        cp_async_point(buf + T::sidx_own(tl, e, l0 + ln), src + (int64_t)(tl + TPL * e) * a.estride);
                }
            }
        }
        cp_async_commit();
    };

    int64_t tile = blockIdx.x;
    stage(tile, buf0, 0);
    stage(tile + gridDim.x, buf1, 1);
    int it = 0;
    bool aborted = false;
    for (; tile < a.ntiles; ++it, tile += gridDim.x) {
        C *sm = (it & 1) ? buf1 : buf0;
        if (tma) {
            // this tile's boxes have landed (the next tile's may still fly)
            const bool ok = mbar_wait_bounded(&mbar[it & 1], (unsigned)(it >> 1) & 1u);
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
        } else {
            cp_async_wait<1>();      // this tile's copies are done (the next tile's may still fly)
            __syncthreads();
        }
        LineGeom g[LPT];
#pragma unroll
        for (int ln = 0; ln < LPT; ++ln) g[ln] = line_geom<L>(a, tile, l0 + ln);
        C v[LPT][E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (tma) T::ld_plain(sm, tl, e, l0, v);    // the copy engine's tile is unswizzled
            else T::ld(sm, tl, e, l0, v);
        }
#pragma unroll
        for (int ln = 0; ln < LPT; ++ln)
            if (!g[ln].valid)
#pragma unroll
                for (int e = 0; e < E; ++e) v[ln][e] = mk((R)0, (R)0);

        if (rmode == RED_DIAG_X || rmode == RED_DIAG_XM) {
            // real-space moments of rho = |psi|^2 along each row, then kx^2 |F_x psi|^2
            // (RED_DIAG_XM, for rms sizes: the moments only)
            const R lox = (R)a.lo[0], hx = (R)a.h[0];
            const R *vsd = static_cast<const R *>(a.vsamp_diag);
            R s0[LPT], sx2[LPT], s4[LPT], sv[LPT];
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) {
                s0[ln] = sx2[ln] = s4[ln] = sv[ln] = (R)0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const R x = lox + (R)(tl + TPL * e) * hx;
                    const R rho = cabs2(v[ln][e]);
                    s0[ln] += rho;
                    sx2[ln] += x * x * rho;
                    s4[ln] += rho * rho;
                    if (vsd) sv[ln] += vsd[g[ln].off + (int64_t)(tl + TPL * e) * a.estride] * rho;
                }
            }
            R sk[LPT];
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) sk[ln] = (R)0;
            if (rmode == RED_DIAG_X) {
                T::template fft<-1, PING>(v, sm, PING ? scr : sm, tl, l0, tw);
                const R kf = (R)a.kf[0];
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int i = tl + TPL * e;
                        const R k = kf * (R)(i < N / 2 ? i : i - N);
                        sk[ln] += k * k * cabs2(v[ln][e]);
                    }
                }
            }
            // the per-line quantities: 0 rho, 1 x^2 rho, 2 y^2 rho, 3 z^2 rho,
            // 4 V rho, 5 rho^2, 6 kx^2 |F_x psi|^2 (y, z, V_y + V_z are constant along the row)
            auto line_q = [&](int ln, int k, double ls0, double lsx2, double ls4, double lsv, double lsk) {
                const int ti = g[ln].ti;
                const double y = a.lo[1] + (double)g[ln].c0 * a.h[1], z = a.lo[2] + (double)g[ln].c1 * a.h[2];
                const double gx = a.gamma[3 * ti + 0], gy = a.gamma[3 * ti + 1], gz = a.gamma[3 * ti + 2];
                const double vyz = 0.5 * gy * gy * y * y + 0.5 * gz * gz * z * z;
                return k == 0 ? ls0
                       : k == 1 ? lsx2
                       : k == 2 ? y * y * ls0
                       : k == 3 ? z * z * ls0
                       : k == 4 ? 0.5 * gx * gx * lsx2 + vyz * ls0 + lsv
                       : k == 5 ? ls4
                                : lsk;
            };
            if constexpr (sizeof(R) == 4) {
                // complex64: the five row sums in double-float, the products by the
                // row's constants in double once per row (FP64 is slow here)
                float qh[5][LPT], ql[5][LPT];
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) {
                    qh[0][ln] = s0[ln];
                    qh[1][ln] = sx2[ln];
                    qh[2][ln] = s4[ln];
                    qh[3][ln] = sv[ln];
                    qh[4][ln] = sk[ln];
#pragma unroll
                    for (int k = 0; k < 5; ++k) ql[k][ln] = 0.0f;
                }
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    group_sum_df<L, TPL, LPT>(qh[k], ql[k], reinterpret_cast<float2 *>(red), l0, tl);
                if (tl == 0) {
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln) {
                        if (!g[ln].valid) continue;
                        const double ls0 = (double)qh[0][ln] + (double)ql[0][ln];
                        const double lsx2 = (double)qh[1][ln] + (double)ql[1][ln];
                        const double ls4 = (double)qh[2][ln] + (double)ql[2][ln];
                        const double lsv = (double)qh[3][ln] + (double)ql[3][ln];
                        const double lsk = (double)qh[4][ln] + (double)ql[4][ln];
                        // the row's constants once (FP64 instructions are what this costs)
                        const int ti = g[ln].ti;
                        const double y = fma((double)g[ln].c0, a.h[1], a.lo[1]);
                        const double z = fma((double)g[ln].c1, a.h[2], a.lo[2]);
                        const double y2 = y * y, z2 = z * z;
                        const double gx = a.gamma[3 * ti + 0], gy = a.gamma[3 * ti + 1], gz = a.gamma[3 * ti + 2];
                        const double vyz = 0.5 * fma(gy * gy, y2, gz * gz * z2);
                        double *pp = a.partials + g[ln].lg;
                        const int64_t cap = a.lines_cap;
                        pp[0] = ls0;
                        pp[cap] = lsx2;
                        pp[2 * cap] = y2 * ls0;
                        pp[3 * cap] = z2 * ls0;
                        pp[4 * cap] = fma(0.5 * gx * gx, lsx2, fma(vyz, ls0, lsv));
                        pp[5 * cap] = ls4;
                        pp[6 * cap] = lsk;
                    }
                }
            } else {
                double q[7][LPT];
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) {
#pragma unroll
                    for (int k = 0; k < 7; ++k)
                        q[k][ln] = line_q(ln, k, (double)s0[ln], (double)sx2[ln], (double)s4[ln], (double)sv[ln],
                                          (double)sk[ln]);
                }
#pragma unroll 1
                for (int k = 0; k < 7; ++k) {
                    group_sum<L, TPL, LPT>(q[k], red, l0, tl);
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln)
                        if (tl == 0 && g[ln].valid) a.partials[(int64_t)k * a.lines_cap + g[ln].lg] = q[k][ln];
                }
            }
        } else if (rmode == RED_DIAG_K) {
            T::template fft<-1, PING>(v, sm, PING ? scr : sm, tl, l0, tw);
            const R kf = (R)a.kf[a.axis];
            R acc[LPT];
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) {
                acc[ln] = (R)0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = tl + TPL * e;
                    const R k = kf * (R)(i < N / 2 ? i : i - N);
                    acc[ln] += k * k * cabs2(v[ln][e]);
                }
            }
            double sk[LPT];
            if constexpr (sizeof(R) == 4) {
                float lo[LPT];
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) lo[ln] = 0.0f;
                group_sum_df<L, TPL, LPT>(acc, lo, reinterpret_cast<float2 *>(red), l0, tl);
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) sk[ln] = (double)acc[ln] + (double)lo[ln];
            } else {
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln) sk[ln] = (double)acc[ln];
                group_sum<L, TPL, LPT>(sk, red, l0, tl);
            }
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln)
                if (tl == 0 && g[ln].valid) a.partials[(int64_t)(6 + a.axis) * a.lines_cap + g[ln].lg] = sk[ln];
        } else {
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln)
                point_op<R, E, TPL>(op_pre, v[ln], a, g[ln].inst, g[ln].ti, g[ln].c0, g[ln].c1, tl, g[ln].off);
            sweep_transforms<T, PING>(v, sm, PING ? scr : sm, tl, l0, tw, fft1, fft2, [&]() {
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln)
                    point_op<R, E, TPL>(op_mid, v[ln], a, g[ln].inst, g[ln].ti, g[ln].c0, g[ln].c1, tl, g[ln].off);
            });
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln)
                point_op<R, E, TPL>(op_post, v[ln], a, g[ln].inst, g[ln].ti, g[ln].c0, g[ln].c1, tl, g[ln].off);
            if (rmode == RED_NORM) {
                if constexpr (sizeof(R) == 4) {
                    float nh[LPT], nl[LPT];
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln) {
                        nh[ln] = 0.0f;
                        nl[ln] = 0.0f;
#pragma unroll
                        for (int e = 0; e < E; ++e) df_acc(nh[ln], nl[ln], cabs2(v[ln][e]));
                    }
                    group_sum_df<L, TPL, LPT>(nh, nl, reinterpret_cast<float2 *>(red), l0, tl);
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln)
                        if (tl == 0 && g[ln].valid) a.partials[g[ln].lg] = (double)nh[ln] + (double)nl[ln];
                } else {
                    double sn[LPT];
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln) {
                        sn[ln] = 0.0;
#pragma unroll
                        for (int e = 0; e < E; ++e) sn[ln] += (double)cabs2(v[ln][e]);
                    }
                    group_sum<L, TPL, LPT>(sn, red, l0, tl);
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln)
                        if (tl == 0 && g[ln].valid) a.partials[g[ln].lg] = sn[ln];
                }
            }
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) {
                if (g[ln].valid) {
                    C *dst = inst_dst<C>(a, g[ln].inst) + g[ln].off;
#pragma unroll
                    for (int e = 0; e < E; ++e) dst[(int64_t)(tl + TPL * e) * a.estride] = v[ln][e];
                }
            }
        }
        if (tma) fence_async_shared();   // this thread's accesses to the buffer precede the next copy into it
        __syncthreads();         // every thread is done with this buffer
        stage(tile + 2 * (int64_t)gridDim.x, sm, it & 1);
    }
    // this CTA's tiles are written: the next kernel may start its launch (its
    // CTAs still wait for this whole grid before they read the state)
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
    if (!tma) {
        cp_async_wait<0>();
    } else if (aborted && t == 0) {
        // report, then let the boxes still in flight land before the CTA exits
        if (a.err) atomicOr(a.err, (int)ERR_TMA_TIMEOUT);
        for (int b = 0; b < 2; ++b) {
            int waited = b == 0 ? (it + 1) / 2 : it / 2;
            for (; waited < issued[b]; ++waited)
                if (!mbar_wait_bounded(&mbar[b], (unsigned)waited & 1u)) break;
        }
    }
}

// ------------------------------------------------------------------ 1D on chip
__host__ __device__ constexpr size_t line1d_red_bytes(int nt) { return (sizeof(double) * (size_t)nt + 15) / 16 * 16; }

// Each line is one instance and stays in registers for all nsteps steps of
// the launch; real time merges consecutive nonlinear half-steps, imaginary
// time renormalises the line after every step.
template <typename R, int N, int L>
__global__ void __launch_bounds__(Tile<R, N, L, true>::NT) k_line1d(const Line1DArgs a)
{
    using T = Tile<R, N, L, true>;
    using C = typename T::C;
    constexpr int E = T::E, TPL = T::TPL;
    using U = typename T::U;
    if (a.stop && *reinterpret_cast<const volatile int *>(a.stop)) return;   // see k_pass
    extern __shared__ __align__(128) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    double *red = reinterpret_cast<double *>(smraw + sizeof(C) * T::SMEM_POINTS);
    // the reduction scratch is rounded up to 16 bytes so that the 16-byte
    // twiddle entries after it stay aligned (tiles of one short line have an
    // odd thread count)
    U *tw = reinterpret_cast<U *>(smraw + sizeof(C) * T::SMEM_POINTS + line1d_red_bytes(T::NT));
    const int t = threadIdx.x, l = T::line_of(t), tl = T::tl_of(t);
    for (int i = t; i < N; i += T::NT) tw[i] = static_cast<const U *>(a.tw)[i];
    __syncthreads();
    const int64_t ntiles = (a.batch + L - 1) / L;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t inst = tile * L + l;
        const bool valid = inst < a.batch;
        const int64_t ip = valid ? inst : 0;
        // instance storage and its parameter/table slot
        C *psi = a.inst_ptr ? static_cast<C *>(a.inst_ptr[ip]) : static_cast<C *>(a.psi) + ip * N;
        const int64_t ib = a.slot_of ? a.slot_of[ip] : ip;
        C v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = valid ? psi[tl + TPL * e] : mk((R)0, (R)0);
        const double g = a.g[ib];
        if (!a.imag) {
            const U *kt = static_cast<const U *>(a.kt);
            const U *vh = static_cast<const U *>(a.vh);
            const U *vf = static_cast<const U *>(a.vf);
            const R gh = (R)(g * 0.5 * a.dt), gf = (R)(g * a.dt);
            const R invn = (R)(1.0 / N);
            // first nonlinear half-step
            {
                R th[E];
#pragma unroll
                for (int e = 0; e < E; ++e) th[e] = gh * cabs2(v[e]);
                apply_phase<C, R, E>(v, th);
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (vh) v[e] = uomul(v[e], vh[ib * N + tl + TPL * e]);
#pragma unroll 1
            for (int64_t st = 0; st < a.nsteps; ++st) {
                T::template fft<-1>(v, sm, tl, l, tw);
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = cscale(uomul(v[e], kt[tl + TPL * e]), invn);
                T::template fft<1>(v, sm, tl, l, tw);
                const bool last = (st == a.nsteps - 1);
                const R gc = last ? gh : gf;
                const U *vt = last ? (a.vh_last ? static_cast<const U *>(a.vh_last) : vh) : vf;
                R th[E];
#pragma unroll
                for (int e = 0; e < E; ++e) th[e] = gc * cabs2(v[e]);
                apply_phase<C, R, E>(v, th);
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (vt) v[e] = uomul(v[e], vt[ib * N + tl + TPL * e]);
            }
        } else {
            const R *ki = static_cast<const R *>(a.kt);
            const R *vi = static_cast<const R *>(a.vi);
            const R gh = (R)(g * 0.5 * a.dt);
            R sc = (R)1;
#pragma unroll 1
            for (int64_t st = 0; st < a.nsteps; ++st) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    C x = cscale(v[e], sc);
                    R f = exp_r(-gh * cabs2(x));
                    if (vi) f *= vi[ib * N + tl + TPL * e];
                    v[e] = cscale(x, f);
                }
                T::template fft<-1>(v, sm, tl, l, tw);
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = cscale(v[e], ki[tl + TPL * e]);
                T::template fft<1>(v, sm, tl, l, tw);
                double nrm = 0.0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    R f = exp_r(-gh * cabs2(v[e]));
                    if (vi) f *= vi[ib * N + tl + TPL * e];
                    v[e] = cscale(v[e], f);
                    nrm += (double)cabs2(v[e]);
                }
                nrm = line_sum<L, TPL>(nrm, red, l, tl);
                if (!(nrm > 0.0) || !isfinite(nrm)) {
                    if (valid && tl == 0) atomicOr(a.err, (int)ERR_NUMERIC);
                    sc = (R)1;
                } else {
                    sc = (R)sqrt(a.target_norm_over_dv / nrm);
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cscale(v[e], sc);
        }
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) psi[tl + TPL * e] = v[e];
        }
    }
}

// ------------------------------------------------------------------ dispatch
struct LaunchCache {
    std::mutex mu;
    int grid_cap[64] = {0};   // per device
};

template <typename K>
static cudaError_t prepare(K kern, LaunchCache &lc, int nt, size_t smem, int *cap)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(lc.mu);
    if (!lc.grid_cap[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nt, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        lc.grid_cap[dev] = nb * sms;
    }
    *cap = lc.grid_cap[dev];
    return cudaSuccess;
}

template <typename R, int N, bool ROWS, int VAR, int PROG>
static cudaError_t launch_pass_p(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    constexpr int L = pick_lines<R, N, ROWS, VAR>();
    using T = PassTile<R, N, ROWS, VAR>;
    static_assert(T::layout_consistent(), "shared layout of the exchanges");
    static LaunchCache lc;
    static const CUtensorMap none = {};
    const size_t smem = pass_smem_bytes<R, N, ROWS, VAR>();
    if (a.tma_chunks > 0 && (ROWS || !tmap || (int64_t)a.tma_chunks * a.tma_box != N || a.tma_box > 256 ||
                             a.axis < 1 || a.o0n % L != 0))
        return cudaErrorInvalidValue;
    int cap = 0;
    cudaError_t e = prepare(k_pass<R, N, ROWS, VAR, PROG>, lc, T::NT, smem, &cap);
    if (e != cudaSuccess) return e;
    if (a.ntiles <= 0) return cudaSuccess;
    const int grid = (int)(a.ntiles < cap ? a.ntiles : cap);
    // launched with programmatic stream serialisation: the kernel waits for
    // its predecessor in the stream itself (griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(T::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pass<R, N, ROWS, VAR, PROG>, a, tmap ? *tmap : none);
}

// complex64 lines of 256 to 1024 points (the large grids) get the fixed-program
// kernels of the sweeps they run; everything else the generic one
template <typename R, int N, bool ROWS> constexpr bool sweep_progs_compiled()
{
    return sizeof(R) == 4 && N >= 256 && N <= 1024;
}
template <typename R, int N, bool ROWS, int VAR>
static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    if constexpr (sweep_progs_compiled<R, N, ROWS>()) {
        const int p = sweep_prog_of(a);
        if constexpr (ROWS) {
            if (p == 4) return launch_pass_p<R, N, ROWS, VAR, 4>(a, st, tmap);
            if (p == 5) return launch_pass_p<R, N, ROWS, VAR, 5>(a, st, tmap);
            if (p == 7) return launch_pass_p<R, N, ROWS, VAR, 7>(a, st, tmap);
            if (p == 8) return launch_pass_p<R, N, ROWS, VAR, 8>(a, st, tmap);
            if (p == 9) return launch_pass_p<R, N, ROWS, VAR, 9>(a, st, tmap);
        } else {
            if (p == 1) return launch_pass_p<R, N, ROWS, VAR, 1>(a, st, tmap);
            if (p == 2) return launch_pass_p<R, N, ROWS, VAR, 2>(a, st, tmap);
            if (p == 3) return launch_pass_p<R, N, ROWS, VAR, 3>(a, st, tmap);
            if (p == 6) return launch_pass_p<R, N, ROWS, VAR, 6>(a, st, tmap);
        }
    }
    return launch_pass_p<R, N, ROWS, VAR, 0>(a, st, tmap);
}

static int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

template <typename R, int N, int L> static cudaError_t launch_line1d_l(const Line1DArgs &a, cudaStream_t st)
{
    using T = Tile<R, N, L, true>;
    static LaunchCache lc;
    const size_t smem = sizeof(typename T::C) * T::SMEM_POINTS + line1d_red_bytes(T::NT) + sizeof(typename T::U) * N;
    int cap = 0;
    cudaError_t e = prepare(k_line1d<R, N, L>, lc, T::NT, smem, &cap);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (a.batch + L - 1) / L;
    if (ntiles <= 0) return cudaSuccess;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    k_line1d<R, N, L><<<grid, T::NT, smem, st>>>(a);
    return cudaGetLastError();
}

// Fewer instances than SMs: one line per CTA, so that no warp spends the SM's
// pipes on the empty lines of a part-filled tile (the per-line arithmetic is
// the same either way).
template <typename R, int N> static cudaError_t launch_line1d_t(const Line1DArgs &a, cudaStream_t st)
{
    constexpr int L = pick_lines_1d<R, N>();
    if constexpr (L > 1) {
        if (a.batch < sm_count()) return launch_line1d_l<R, N, 1>(a, st);
    }
    return launch_line1d_l<R, N, L>(a, st);
}

#define GPE_FOR_EACH_N(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

// Strided complex64 lines of 256 to 1024 points (radix-32 kernels, the
// longest to compile) are instantiated in translation units of their own,
// one per line length and tile shape (pass_f32_w<N>_<VAR>.cu), so that the
// library builds in parallel.
template <int N, int VAR> cudaError_t launch_pass_wide_f32(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap);
template <typename R, int N, bool ROWS> constexpr bool pass_wide_tu()
{
    return sizeof(R) == 4 && !ROWS && N >= 256 && N <= 1024;
}
template <typename R, int N, bool ROWS, int VAR>
static cudaError_t launch_pass_n(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    if constexpr (pass_wide_tu<R, N, ROWS>()) return launch_pass_wide_f32<N, VAR>(a, st, tmap);
    else return launch_pass_t<R, N, ROWS, VAR>(a, st, tmap);
}

template <typename R, bool ROWS, int VAR>
static cudaError_t launch_pass_r(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    switch (a.nax) {
#define GPE_CASE(NN) \
    case NN: return launch_pass_n<R, NN, ROWS, VAR>(a, st, tmap);
        GPE_FOR_EACH_N(GPE_CASE)
#undef GPE_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename R> static int lines_per_tile_r(bool rows, int n, int var)
{
    switch (n) {
#define GPE_CASE(NN)                                                                                 \
    case NN:                                                                                         \
        return rows ? (var ? pick_lines<R, NN, true, 1>() : pick_lines<R, NN, true, 0>())            \
                    : (var ? pick_lines<R, NN, false, 1>() : pick_lines<R, NN, false, 0>());
        GPE_FOR_EACH_N(GPE_CASE)
#undef GPE_CASE
    default: return 0;
    }
}

template <typename R> static cudaError_t launch_line1d_r(const Line1DArgs &a, cudaStream_t st)
{
    switch (a.n) {
#define GPE_CASE(NN) \
    case NN: return launch_line1d_t<R, NN>(a, st);
        GPE_FOR_EACH_N(GPE_CASE)
#undef GPE_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe
