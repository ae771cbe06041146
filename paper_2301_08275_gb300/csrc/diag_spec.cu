// diag_spec.cu - FP64 reductions (norm, energy, mu, rms sizes, renormalisation
// factor) and the kernels of the kinetic-energy spectra.
#include <math.h>

#include "fft_tile.cuh"
#include <algorithm>

#include "gpe_internal.h"

namespace gpe {

// ------------------------------------------------------------------ reductions
// sums[b*NQ + q] = sum over the lines of instance b of partials[q][line], in a
// fixed order that depends only on the number of lines: chunks of
// REDUCE_CHUNK consecutive lines are summed by one CTA each (strided
// per-thread sums into four accumulators, warp shuffles, one shared-memory
// stage), then one warp per (instance, quantity) adds the chunk sums (strided
// per lane, shuffles).  FP64 additions are slow on this GPU (one warp
// instruction per 64 cycles per SM sub-partition): spreading them over many
// SMs is what makes the sum fast (65536 lines: 24 us in one CTA before).
__global__ void __launch_bounds__(256) k_reduce_chunks(const double *__restrict__ partials, int64_t cap, int q0,
                                                       int64_t lpi, int64_t nch, double *__restrict__ csum,
                                                       const int *stop)
{
    __shared__ double sh[8];
    if (stop && *reinterpret_cast<const volatile int *>(stop)) return;
    const int64_t c = blockIdx.x, b = blockIdx.z;
    const int q = q0 + blockIdx.y, t = threadIdx.x;
    const int64_t first = c * REDUCE_CHUNK;
    const int64_t n = lpi - first < REDUCE_CHUNK ? lpi - first : REDUCE_CHUNK;
    const double *p = partials + (int64_t)q * cap + b * lpi + first;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t j = t;
    for (; j + 3 * 256 < n; j += 4 * 256) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += p[j + (int64_t)k * 256];
    }
    for (int k = 0; j < n; j += 256, ++k) acc[k & 3] += p[j];
    double s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((t & 31) == 0) sh[t >> 5] = s;
    __syncthreads();
    if (t == 0) {
        const double r = ((sh[0] + sh[1]) + (sh[2] + sh[3])) + ((sh[4] + sh[5]) + (sh[6] + sh[7]));
        csum[(b * NQ + q) * nch + c] = r;
    }
}

// One warp per (instance, quantity): sums of the chunk sums.  With scale set,
// the sum of quantity 0 (the norm) also gives the imaginary-time
// renormalisation factor s_b = sqrt(target / (sum rho dV)).
__global__ void __launch_bounds__(128) k_reduce_final(const double *__restrict__ csum, int q0, int nq, int64_t batch,
                                                      int64_t nch, double *__restrict__ sums, double dv, double target,
                                                      double *__restrict__ scale, int *err, const int *stop)
{
    if (stop && *reinterpret_cast<const volatile int *>(stop)) return;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= batch * nq) return;      // uniform per warp
    const int64_t b = w / nq;
    const int q = q0 + (int)(w % nq);
    const double *p = csum + (b * NQ + q) * nch;
    double s = 0.0;
    for (int64_t j = lane; j < nch; j += 32) s += p[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        sums[b * NQ + q] = s;
        if (scale && q == 0) {
            const double nrm = s * dv;
            if (!(nrm > 0.0) || !isfinite(nrm)) {
                atomicOr(err, (int)ERR_NUMERIC);
                scale[b] = 1.0;
            } else {
                scale[b] = sqrt(target / nrm);
            }
        }
    }
}

// norm, E_kin, E_pot, E_int, E, mu and sigma_x, sigma_y, sigma_z, r_rms from the
// per-instance sums of the diagnostic passes.
__global__ void k_finish_diag(const double *__restrict__ sums, int64_t batch, int ndim, int64_t n0, int64_t n1,
                              int64_t n2, double dv, const double *__restrict__ g, double *__restrict__ out6,
                              double *__restrict__ out4, const int *stop)
{
    if (stop && *reinterpret_cast<const volatile int *>(stop)) return;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double *q = sums + b * NQ;
    const double nrm = q[0] * dv;
    const double n[3] = {(double)n0, (double)n1, (double)n2};
    double ek = 0.0;
    for (int a = 0; a < ndim; ++a) ek += q[6 + a] / n[a];
    ek *= 0.5 * dv;
    const double ep = q[4] * dv;
    const double ei = 0.5 * g[b] * q[5] * dv;
    out6[6 * b + 0] = nrm;
    out6[6 * b + 1] = ek;
    out6[6 * b + 2] = ep;
    out6[6 * b + 3] = ei;
    out6[6 * b + 4] = ek + ep + ei;
    out6[6 * b + 5] = (ek + ep + 2.0 * ei) / nrm;
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double s2 = a < ndim ? q[1 + a] / q[0] : 0.0;
        out4[4 * b + a] = sqrt(s2);
        r2 += s2;
    }
    out4[4 * b + 3] = sqrt(r2);
}

int64_t reduce_chunks(int64_t lines_per_inst) { return (lines_per_inst + REDUCE_CHUNK - 1) / REDUCE_CHUNK; }

cudaError_t launch_reduce_lines(const double *partials, int64_t lines_cap, int nq_first, int nq, int64_t batch,
                                int64_t lines_per_inst, double *csum, double *sums, cudaStream_t st, double dv,
                                double target, double *scale, int *err, const int *stop)
{
    if (batch <= 0 || nq <= 0) return cudaSuccess;
    const int64_t nch = reduce_chunks(lines_per_inst);
    dim3 grid((unsigned)nch, (unsigned)nq, (unsigned)batch);
    k_reduce_chunks<<<grid, 256, 0, st>>>(partials, lines_cap, nq_first, lines_per_inst, nch, csum, stop);
    const int64_t warps = batch * nq;
    k_reduce_final<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(csum, nq_first, nq, batch, nch, sums, dv, target,
                                                              scale, err, stop);
    return cudaGetLastError();
}

__global__ void k_imag_init(const double *__restrict__ out6, double *__restrict__ eprev, int64_t batch, int *stop,
                            int64_t *done)
{
    for (int64_t b = threadIdx.x; b < batch; b += blockDim.x) eprev[b] = out6[6 * b + 4];
    if (threadIdx.x == 0) {
        *stop = 0;
        *done = 0;
    }
}

__global__ void __launch_bounds__(256) k_imag_check(const double *__restrict__ out6, double *__restrict__ eprev,
                                                    int64_t batch, double etol, int64_t chunk, int *stop,
                                                    int64_t *done, const int *err)
{
    if (*reinterpret_cast<const volatile int *>(stop)) return;
    // the host rule of gpe_step_imag: stop when every instance moved by less
    // than etol since the last check (never for etol <= 0)
    int moved = !(etol > 0.0), bad = 0;
    for (int64_t b = threadIdx.x; b < batch; b += blockDim.x) {
        const double e = out6[6 * b + 4];
        if (!isfinite(e)) bad = 1;
        if (!(fabs(e - eprev[b]) < etol)) moved = 1;
        eprev[b] = e;
    }
    moved = __syncthreads_or(moved);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        *done += chunk;
        if (bad || (err && (*reinterpret_cast<const volatile int *>(err) & ERR_NUMERIC))) *stop = 2;
        else if (!moved) *stop = 1;
    }
}

cudaError_t launch_imag_init(const double *out6, double *eprev, int64_t batch, int *stop, int64_t *done,
                             cudaStream_t st)
{
    k_imag_init<<<1, 256, 0, st>>>(out6, eprev, batch, stop, done);
    return cudaGetLastError();
}

cudaError_t launch_imag_check(const double *out6, double *eprev, int64_t batch, double etol, int64_t chunk, int *stop,
                              int64_t *done, const int *err, cudaStream_t st)
{
    k_imag_check<<<1, 256, 0, st>>>(out6, eprev, batch, etol, chunk, stop, done, err);
    return cudaGetLastError();
}

cudaError_t launch_finish_diag(const double *sums, int64_t batch, int ndim, const int64_t *n, double dv,
                               const double *g, double *out6, double *out4, cudaStream_t st, const int *stop)
{
    const int nb = (int)((batch + 127) / 128);
    k_finish_diag<<<nb, 128, 0, st>>>(sums, batch, ndim, n[0], n[1], n[2], dv, g, out6, out4, stop);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ spectra
__device__ __forceinline__ int64_t axis_index(int64_t i, const SpecArgs &s, int axis)
{
    int64_t stride = 1;
    for (int a = 0; a < axis; ++a) stride *= s.n[a];
    return (i / stride) % s.n[axis];
}

// dst = i k_axis src, with the Nyquist mode of i k_axis set to zero.
template <typename R>
__global__ void k_deriv(const SpecArgs s, const typename CT<R>::C *__restrict__ src, typename CT<R>::C *__restrict__ dst,
                        int axis)
{
    using C = typename CT<R>::C;
    const int64_t na = s.n[axis];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = axis_index(i, s, axis);
        const R k = (2 * j == na) ? (R)0 : (R)(s.kf[axis] * (double)(j < na / 2 ? j : j - na));
        const C v = src[i];
        dst[i] = mk(-k * v.y, k * v.x);
    }
}

// w <- u = Im(conj(psi) * w / N) / |psi| (part 0) or Re(...) / |psi| (part 1: the
// gradient of |psi|), 0 where |psi|^2 < 1e-30, stored as (u, 0).
template <typename R>
__global__ void k_velocity(const SpecArgs s, const typename CT<R>::C *__restrict__ psi, typename CT<R>::C *__restrict__ w)
{
    using C = typename CT<R>::C;
    const R invn = (R)(1.0 / (double)s.N);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.N; i += (int64_t)gridDim.x * blockDim.x) {
        const C p = psi[i];
        const C d = w[i];
        const R rho = p.x * p.x + p.y * p.y;
        R u = (R)0;
        if (rho >= (R)1e-30) u = (s.part ? (p.x * d.x + p.y * d.y) : (p.x * d.y - p.y * d.x)) * invn / sqrt(rho);
        w[i] = mk(u, (R)0);
    }
}

// Shell histogram of |u_i|^2 and |u_c|^2 (split) or of sum_a |u_a|^2 (slot 0)
// over the k grid, one partial histogram per block (hist[block][2][nshells]).
// Shell sums are accumulated in 64-bit fixed point so that they do not depend
// on the order in which threads add (integer addition is associative): a
// deterministic pre-pass sums |u|^2 over the field in a fixed tree order,
// the scale is the power of two that maps that total below 2^62, and every
// point's contribution is rounded to an integer multiple of 1/scale before
// the (integer) atomic additions.  Rounding costs at most total * 2^-63 per
// point; the errors are of either sign and far below the FP64 sums' own.
template <typename R>
__global__ void k_field_total(const SpecArgs s, const typename CT<R>::C *__restrict__ u0,
                              const typename CT<R>::C *__restrict__ u1, const typename CT<R>::C *__restrict__ u2,
                              double *__restrict__ partial)
{
    using C = typename CT<R>::C;
    __shared__ double red[256];
    const C *u[3] = {u0, u1, u2};
    const int nc = s.split ? s.ndim : s.ncomp;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.N; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < nc; ++a) {
            const C v = u[a][i];
            acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}
// fixed-order sum of the block partials; scale = 2^(61 - ceil(log2 total))
__global__ void k_fixed_scale(double *aux, int nblocks)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += aux[b];
    int ex = 0;
    frexp(t > 0.0 ? t : 1.0, &ex);               // t < 2^ex
    aux[nblocks] = ldexp(1.0, 61 - ex);
}

template <typename R>
__global__ void k_bin(const SpecArgs s, const typename CT<R>::C *__restrict__ u0, const typename CT<R>::C *__restrict__ u1,
                      const typename CT<R>::C *__restrict__ u2, int64_t nshells, const double *__restrict__ scale_p,
                      unsigned long long *__restrict__ hist)
{
    using C = typename CT<R>::C;
    extern __shared__ unsigned long long shq[];   // [2][nshells]
    for (int64_t i = threadIdx.x; i < 2 * nshells; i += blockDim.x) shq[i] = 0ull;
    __syncthreads();
    const double scale = *scale_p;
    auto fx = [scale](double v) { return (unsigned long long)(v * scale + 0.5); };
    const C *u[3] = {u0, u1, u2};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.N; i += (int64_t)gridDim.x * blockDim.x) {
        double kv[3] = {0.0, 0.0, 0.0}, q2 = 0.0, k2 = 0.0;
        int64_t rem = i;
        for (int a = 0; a < s.ndim; ++a) {
            const int64_t j = rem % s.n[a];
            rem /= s.n[a];
            const int64_t m = j < s.n[a] / 2 ? j : j - s.n[a];
            kv[a] = s.kf[a] * (double)m;
            k2 += kv[a] * kv[a];
            const double qa = (double)m * s.lratio[a];
            q2 += qa * qa;
        }
        const int64_t sh_i = (int64_t)floor(sqrt(q2) + 0.5);
        if (!s.split) {
            double et = 0.0;
            for (int a = 0; a < s.ncomp; ++a) {
                const C v = u[a][i];
                et += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            }
            atomicAdd(&shq[sh_i], fx(et));
            continue;
        }
        double ur[3] = {0, 0, 0}, ui[3] = {0, 0, 0}, kdr = 0.0, kdi = 0.0;
        for (int a = 0; a < s.ndim; ++a) {
            const C v = u[a][i];
            ur[a] = (double)v.x;
            ui[a] = (double)v.y;
            kdr += kv[a] * ur[a];
            kdi += kv[a] * ui[a];
        }
        double ec = 0.0, ei = 0.0;
        for (int a = 0; a < s.ndim; ++a) {
            const double cr = k2 > 0.0 ? kv[a] * kdr / k2 : 0.0;
            const double ci = k2 > 0.0 ? kv[a] * kdi / k2 : 0.0;
            ec += cr * cr + ci * ci;
            ei += (ur[a] - cr) * (ur[a] - cr) + (ui[a] - ci) * (ui[a] - ci);
        }
        atomicAdd(&shq[sh_i], fx(ei));
        atomicAdd(&shq[nshells + sh_i], fx(ec));
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < 2 * nshells; i += blockDim.x) hist[(int64_t)blockIdx.x * 2 * nshells + i] = shq[i];
}
__global__ void k_hist_reduce(const unsigned long long *__restrict__ hist, int nblocks, int64_t nshells,
                              const double *__restrict__ scale_p, double half_dv_over_n, double *__restrict__ out_inc,
                              double *__restrict__ out_comp)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nshells) return;
    unsigned long long a = 0ull, c = 0ull;
    for (int b = 0; b < nblocks; ++b) {
        a += hist[(int64_t)b * 2 * nshells + s];
        c += hist[(int64_t)b * 2 * nshells + nshells + s];
    }
    const double inv = 1.0 / *scale_p;            // a power of two: exact
    out_inc[s] = half_dv_over_n * ((double)a * inv);
    out_comp[s] = half_dv_over_n * ((double)c * inv);
}

static int grid_for(int64_t N)
{
    int64_t b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

int bin_blocks(const SpecArgs &s)
{
    int64_t b = (s.N + 255) / 256;
    if (b > 152 * 2) b = 152 * 2;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_deriv(const SpecArgs &s, const void *src, void *dst, int axis, cudaStream_t st)
{
    if (s.prec == 0)
        k_deriv<float><<<grid_for(s.N), 256, 0, st>>>(s, (const float2 *)src, (float2 *)dst, axis);
    else
        k_deriv<double><<<grid_for(s.N), 256, 0, st>>>(s, (const double2 *)src, (double2 *)dst, axis);
    return cudaGetLastError();
}

cudaError_t launch_velocity(const SpecArgs &s, const void *psi, void *w, cudaStream_t st)
{
    if (s.prec == 0)
        k_velocity<float><<<grid_for(s.N), 256, 0, st>>>(s, (const float2 *)psi, (float2 *)w);
    else
        k_velocity<double><<<grid_for(s.N), 256, 0, st>>>(s, (const double2 *)psi, (double2 *)w);
    return cudaGetLastError();
}

// Trap tables of one time level (see launch_trap_level): angles in double
// precision from the same formula as the plan's static tables, split into
// hi + lo floats for complex64.
__global__ void k_trap_level(int prec, void *t0, void *t1, void *t2, int ndim, int64_t n0, int64_t n1, int64_t n2,
                             double lo0, double lo1, double lo2, double h0, double h1, double h2, double g0, double g1,
                             double g2, double c, int64_t batch)
{
    const int64_t tot = n0 + (ndim > 1 ? n1 : 0) + (ndim > 2 ? n2 : 0);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot * batch;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = q / tot;
        int64_t j = q - b * tot;
        int a = 0;
        if (j >= n0) {
            j -= n0;
            a = 1;
            if (j >= n1) {
                j -= n1;
                a = 2;
            }
        }
        const int64_t na = a == 0 ? n0 : (a == 1 ? n1 : n2);
        const double x = (a == 0 ? lo0 : (a == 1 ? lo1 : lo2)) + (double)j * (a == 0 ? h0 : (a == 1 ? h1 : h2));
        const double gm = a == 0 ? g0 : (a == 1 ? g1 : g2);
        const double th = 0.5 * gm * gm * x * x * c;
        const double sh = sin(0.5 * th);
        const double wx = -2.0 * sh * sh, wy = -sin(th);
        void *t = a == 0 ? t0 : (a == 1 ? t1 : t2);
        if (prec == 0) {
            const float hx = (float)wx, hy = (float)wy;
            static_cast<float4 *>(t)[b * na + j] =
                make_float4(hx, hy, (float)(wx - (double)hx), (float)(wy - (double)hy));
        } else {
            static_cast<double2 *>(t)[b * na + j] = make_double2(wx, wy);
        }
    }
}

cudaError_t launch_trap_level(int prec, void *const *tab, int ndim, const int64_t *n, const double *lo,
                              const double *h, const double *gamma, double c, int64_t batch, cudaStream_t st)
{
    const int64_t tot = (n[0] + (ndim > 1 ? n[1] : 0) + (ndim > 2 ? n[2] : 0)) * batch;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 1024);
    k_trap_level<<<blocks, 256, 0, st>>>(prec, tab[0], ndim > 1 ? tab[1] : nullptr, ndim > 2 ? tab[2] : nullptr, ndim,
                                         n[0], ndim > 1 ? n[1] : 1, ndim > 2 ? n[2] : 1, lo[0], lo[1], lo[2], h[0], h[1],
                                         h[2], gamma[0], gamma[1], gamma[2], c, batch);
    return cudaGetLastError();
}

cudaError_t launch_bin(const SpecArgs &s, void *const *uh, int64_t nshells, double *block_hist, int nblocks,
                       double *aux, cudaStream_t st)
{
    const size_t smem = sizeof(unsigned long long) * 2 * (size_t)nshells;
    unsigned long long *hq = reinterpret_cast<unsigned long long *>(block_hist);
    cudaError_t e;
    if (s.prec == 0) {
        k_field_total<float><<<nblocks, 256, 0, st>>>(s, (const float2 *)uh[0], (const float2 *)uh[1],
                                                      (const float2 *)uh[2], aux);
        k_fixed_scale<<<1, 32, 0, st>>>(aux, nblocks);
        e = cudaFuncSetAttribute(k_bin<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_bin<float><<<nblocks, 256, smem, st>>>(s, (const float2 *)uh[0], (const float2 *)uh[1],
                                                 (const float2 *)uh[2], nshells, aux + nblocks, hq);
    } else {
        k_field_total<double><<<nblocks, 256, 0, st>>>(s, (const double2 *)uh[0], (const double2 *)uh[1],
                                                       (const double2 *)uh[2], aux);
        k_fixed_scale<<<1, 32, 0, st>>>(aux, nblocks);
        e = cudaFuncSetAttribute(k_bin<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_bin<double><<<nblocks, 256, smem, st>>>(s, (const double2 *)uh[0], (const double2 *)uh[1],
                                                  (const double2 *)uh[2], nshells, aux + nblocks, hq);
    }
    return cudaGetLastError();
}

cudaError_t launch_hist_reduce(const double *block_hist, int nblocks, int64_t nshells, double dv_over_n,
                               const double *aux, double *out_inc, double *out_comp, cudaStream_t st)
{
    const int nb = (int)((nshells + 127) / 128);
    k_hist_reduce<<<nb, 128, 0, st>>>(reinterpret_cast<const unsigned long long *>(block_hist), nblocks, nshells,
                                      aux + nblocks, 0.5 * dv_over_n, out_inc, out_comp);
    return cudaGetLastError();
}

}  // namespace gpe
