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

// exp(-i th) - 1 = (-2 sin^2(th/2), -sin th), from the half angle so that the
// offset keeps full relative precision for small th
template <typename R> __device__ __forceinline__ typename CT<R>::C phase_offset(R th)
{
    R s, c;
    sincos_r((R)0.5 * th, &s, &c);
    return mk((R)-2 * s * s, (R)-2 * s * c);
}

// lines per tile: tile <= 8192 points (complex64) / 4096 (complex128) and
// <= 1024 threads; strided tiles take 16 (c64) / 8 (c128) adjacent lines so
// that every row segment is 128 bytes.
template <typename R, int N, bool ROWS> constexpr int pick_lines()
{
    constexpr int maxpts = sizeof(R) == 4 ? 8192 : 4096;
    constexpr int lmax = ROWS ? 16 : (sizeof(R) == 4 ? 16 : 8);
    int L = maxpts / N;
    if (L > lmax) L = lmax;
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

// pointwise substep on the E points (indices tl + TPL*e on this axis) of one line
template <typename R, int E, int TPL>
__device__ __forceinline__ void point_op(int op, typename CT<R>::C (&v)[E], const PassArgs &a, int inst,
                                         int c0, int c1, int tl)
{
    using C = typename CT<R>::C;
    if (op == OP_NONE) return;
    using U = typename UT<R>::U;
    if (op == OP_KREAL) {
        // tables hold exp(-i k_a^2 dt/2) - 1; the 1/N of the inverse transform is exact
        const U *kt = static_cast<const U *>(a.kt_ax);
        const U *k0 = static_cast<const U *>(a.kt_o0);
        const U *k1 = static_cast<const U *>(a.kt_o1);
        const U f0 = k0 ? k0[c0] : U{}, f1 = k1 ? k1[c1] : U{};
        const R invn = (R)a.inv_n;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C x = uomul(v[e], kt[tl + TPL * e]);
            if (k0) x = uomul(x, f0);
            if (k1) x = uomul(x, f1);
            v[e] = cscale(x, invn);
        }
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
    const R gc = (R)(a.g[inst] * a.nl_c);
    if (op == OP_NREAL) {
        // trap tables hold exp(-i V_a c) - 1
        const U *vax = static_cast<const U *>(a.vt_ax);
        const U *v0 = static_cast<const U *>(a.vt_o0);
        const U *v1 = static_cast<const U *>(a.vt_o1);
        const U f0 = v0 ? v0[(int64_t)inst * a.o0n + c0] : U{};
        const U f1 = v1 ? v1[(int64_t)inst * a.o1n + c1] : U{};
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C x = cmadd1(v[e], phase_offset(gc * cabs2(v[e])));
            if (vax) x = uomul(x, vax[(int64_t)inst * a.nax + tl + TPL * e]);
            if (v0) x = uomul(x, f0);
            if (v1) x = uomul(x, f1);
            v[e] = x;
        }
        return;
    }
    // OP_NIMAG / OP_SCALE_NIMAG
    const R *iax = static_cast<const R *>(a.vi_ax);
    R fl = (R)1;
    if (a.vi_o0) fl *= static_cast<const R *>(a.vi_o0)[(int64_t)inst * a.o0n + c0];
    if (a.vi_o1) fl *= static_cast<const R *>(a.vi_o1)[(int64_t)inst * a.o1n + c1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        R f = fl * exp_r(-gc * cabs2(v[e]));
        if (iax) f *= iax[(int64_t)inst * a.nax + tl + TPL * e];
        v[e] = cscale(v[e], f);
    }
}

template <typename R, int N, int L, bool ROWS>
__global__ void __launch_bounds__(Tile<R, N, L, ROWS>::NT) k_pass(const PassArgs a)
{
    using T = Tile<R, N, L, ROWS>;
    using C = typename T::C;
    constexpr int E = T::E, TPL = T::TPL;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    double *red = reinterpret_cast<double *>(smraw + sizeof(C) * T::SMEM_POINTS);
    const int t = threadIdx.x, l = T::line_of(t), tl = T::tl_of(t);
    const typename T::U *tw = static_cast<const typename T::U *>(a.tw);
    const C *src = static_cast<const C *>(a.src);
    C *dst = static_cast<C *>(a.dst);
    const int64_t lpi_mask = (int64_t(1) << a.lg_lpi) - 1;
    const int64_t a_mask = (int64_t(1) << a.lg_A) - 1;

    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int64_t lg = tile * L + l;
        const bool valid = lg < a.lines_total;
        const int inst = valid ? int(lg >> a.lg_lpi) : 0;
        const int64_t li = lg & lpi_mask;
        const int c0 = int(li & (a.o0n - 1)), c1 = int(li >> a.lg_o0);
        const int64_t base = inst * a.inst_stride + (li & a_mask) + (li >> a.lg_A) * a.Sb;
        C v[E];
#pragma unroll
        for (int e = 0; e < E; ++e)
            v[e] = valid ? src[base + (int64_t)(tl + TPL * e) * a.estride] : mk((R)0, (R)0);

        if (a.red == RED_DIAG_X) {
            // real-space moments of rho = |psi|^2 along the row, then kx^2 |F_x psi|^2
            const double gx = a.gamma[3 * inst + 0];
            const R lox = (R)a.lo[0], hx = (R)a.h[0];
            R s0 = 0, sx2 = 0, s4 = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const R x = lox + (R)(tl + TPL * e) * hx;
                const R rho = cabs2(v[e]);
                s0 += rho;
                sx2 += x * x * rho;
                s4 += rho * rho;
            }
            T::template fft<-1>(v, sm, tl, l, tw);
            const R kf = (R)a.kf[0];
            R sk = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = tl + TPL * e;
                const R k = kf * (R)(i < N / 2 ? i : i - N);
                sk += k * k * cabs2(v[e]);
            }
            const double y = a.lo[1] + (double)c0 * a.h[1], z = a.lo[2] + (double)c1 * a.h[2];
            const double gy = a.gamma[3 * inst + 1], gz = a.gamma[3 * inst + 2];
            const double vyz = 0.5 * gy * gy * y * y + 0.5 * gz * gz * z * z;
            double q[7];
            q[0] = (double)s0;
            q[1] = (double)sx2;
            q[2] = y * y * (double)s0;
            q[3] = z * z * (double)s0;
            q[4] = 0.5 * gx * gx * (double)sx2 + vyz * (double)s0;
            q[5] = (double)s4;
            q[6] = (double)sk;
#pragma unroll 1
            for (int k = 0; k < 7; ++k) {
                const double s = line_sum<L, TPL>(q[k], red, l, tl);
                if (tl == 0 && valid) a.partials[(int64_t)k * a.lines_cap + lg] = s;
            }
            continue;
        }
        if (a.red == RED_DIAG_K) {
            T::template fft<-1>(v, sm, tl, l, tw);
            const R kf = (R)a.kf[a.axis];
            R sk = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = tl + TPL * e;
                const R k = kf * (R)(i < N / 2 ? i : i - N);
                sk += k * k * cabs2(v[e]);
            }
            const double s = line_sum<L, TPL>((double)sk, red, l, tl);
            if (tl == 0 && valid) a.partials[(int64_t)(6 + a.axis) * a.lines_cap + lg] = s;
            continue;
        }

        point_op<R, E, TPL>(a.op_pre, v, a, inst, c0, c1, tl);
        if (a.fft1 < 0) T::template fft<-1>(v, sm, tl, l, tw);
        else if (a.fft1 > 0) T::template fft<1>(v, sm, tl, l, tw);
        point_op<R, E, TPL>(a.op_mid, v, a, inst, c0, c1, tl);
        if (a.fft2 < 0) T::template fft<-1>(v, sm, tl, l, tw);
        else if (a.fft2 > 0) T::template fft<1>(v, sm, tl, l, tw);
        point_op<R, E, TPL>(a.op_post, v, a, inst, c0, c1, tl);
        if (a.red == RED_NORM) {
            double s = 0.0;
#pragma unroll
            for (int e = 0; e < E; ++e) s += (double)cabs2(v[e]);
            s = line_sum<L, TPL>(s, red, l, tl);
            if (tl == 0 && valid) a.partials[lg] = s;
        }
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) dst[base + (int64_t)(tl + TPL * e) * a.estride] = v[e];
        }
    }
}

// ------------------------------------------------------------------ 1D on chip
// Each line is one instance and stays in registers for all nsteps steps of
// the launch; real time merges consecutive nonlinear half-steps, imaginary
// time renormalises the line after every step.
template <typename R, int N, int L>
__global__ void __launch_bounds__(Tile<R, N, L, true>::NT) k_line1d(const Line1DArgs a)
{
    using T = Tile<R, N, L, true>;
    using C = typename T::C;
    constexpr int E = T::E, TPL = T::TPL;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    double *red = reinterpret_cast<double *>(smraw + sizeof(C) * T::SMEM_POINTS);
    const int t = threadIdx.x, l = T::line_of(t), tl = T::tl_of(t);
    using U = typename T::U;
    const U *tw = static_cast<const U *>(a.tw);
    C *psi = static_cast<C *>(a.psi);
    const int64_t ntiles = (a.batch + L - 1) / L;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t inst = tile * L + l;
        const bool valid = inst < a.batch;
        const int64_t ib = valid ? inst : 0;
        C v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = valid ? psi[ib * N + tl + TPL * e] : mk((R)0, (R)0);
        const double g = a.g[ib];
        if (!a.imag) {
            const U *kt = static_cast<const U *>(a.kt);
            const U *vh = static_cast<const U *>(a.vh);
            const U *vf = static_cast<const U *>(a.vf);
            const R gh = (R)(g * 0.5 * a.dt), gf = (R)(g * a.dt);
            const R invn = (R)(1.0 / N);
            // first nonlinear half-step
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v[e] = cmadd1(v[e], phase_offset(gh * cabs2(v[e])));
                if (vh) v[e] = uomul(v[e], vh[ib * N + tl + TPL * e]);
            }
#pragma unroll 1
            for (int64_t st = 0; st < a.nsteps; ++st) {
                T::template fft<-1>(v, sm, tl, l, tw);
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = cscale(uomul(v[e], kt[tl + TPL * e]), invn);
                T::template fft<1>(v, sm, tl, l, tw);
                const bool last = (st == a.nsteps - 1);
                const R gc = last ? gh : gf;
                const U *vt = last ? vh : vf;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    v[e] = cmadd1(v[e], phase_offset(gc * cabs2(v[e])));
                    if (vt) v[e] = uomul(v[e], vt[ib * N + tl + TPL * e]);
                }
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
                    if (valid && tl == 0) atomicExch(a.err, 1);
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
            for (int e = 0; e < E; ++e) psi[ib * N + tl + TPL * e] = v[e];
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

template <typename R, int N, bool ROWS> static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st)
{
    constexpr int L = pick_lines<R, N, ROWS>();
    using T = Tile<R, N, L, ROWS>;
    static LaunchCache lc;
    const size_t smem = sizeof(typename T::C) * T::SMEM_POINTS + sizeof(double) * T::NT;
    int cap = 0;
    cudaError_t e = prepare(k_pass<R, N, L, ROWS>, lc, T::NT, smem, &cap);
    if (e != cudaSuccess) return e;
    if (a.ntiles <= 0) return cudaSuccess;
    const int grid = (int)(a.ntiles < cap ? a.ntiles : cap);
    k_pass<R, N, L, ROWS><<<grid, T::NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R, int N> static cudaError_t launch_line1d_t(const Line1DArgs &a, cudaStream_t st)
{
    constexpr int L = pick_lines<R, N, true>();
    using T = Tile<R, N, L, true>;
    static LaunchCache lc;
    const size_t smem = sizeof(typename T::C) * T::SMEM_POINTS + sizeof(double) * T::NT;
    int cap = 0;
    cudaError_t e = prepare(k_line1d<R, N, L>, lc, T::NT, smem, &cap);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (a.batch + L - 1) / L;
    if (ntiles <= 0) return cudaSuccess;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    k_line1d<R, N, L><<<grid, T::NT, smem, st>>>(a);
    return cudaGetLastError();
}

#define GPE_FOR_EACH_N(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

template <typename R> static cudaError_t launch_pass_r(bool rows, const PassArgs &a, cudaStream_t st)
{
    switch (a.nax) {
#define GPE_CASE(NN) \
    case NN: return rows ? launch_pass_t<R, NN, true>(a, st) : launch_pass_t<R, NN, false>(a, st);
        GPE_FOR_EACH_N(GPE_CASE)
#undef GPE_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename R> static int lines_per_tile_r(bool rows, int n)
{
    switch (n) {
#define GPE_CASE(NN) \
    case NN: return rows ? pick_lines<R, NN, true>() : pick_lines<R, NN, false>();
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
