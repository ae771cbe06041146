// noalloc.cu - gpe_norm_energy_noalloc: the norm/energy diagnostics with all
// of their scratch in one statically sized device array, for callers that
// must not allocate device memory themselves or through this library.
//
// Who needs it: code that runs under another framework's memory manager
// (which owns every byte of device memory and does not allow raw cudaMalloc),
// and tight loops where cudaMalloc/cudaFree are not acceptable because they
// can synchronise the whole device.  Such a caller can still pass psi and a
// host output buffer; everything else lives in g_noalloc_scratch below.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it (about 2.4 MiB) until the process exits.  In host code its
// name is only a stand-in for the device symbol, never a usable address: every
// call looks up the device address on the current device with
// cudaGetSymbolAddress and passes it to the kernels.  The lookup allocates
// nothing once the module is loaded and is not cached, so a device reset or a
// new primary context between calls leaves no stale address behind.
#include <math.h>
#include <string.h>

#include "../../include/gpe.h"
#include "fft_tile.cuh"
#include "gpe_internal.h"

namespace {

using namespace gpe;

constexpr int64_t kMaxLines = GPE_NOALLOC_MAX_LINES;   // lines per axis (N / n_a)
constexpr int kMaxN = 4096;                             // points per axis

// layout of the scratch array (byte offsets, each region 256-byte aligned)
constexpr size_t kPartialsOff = 0;
constexpr size_t kPartialsBytes = sizeof(double) * NQ * kMaxLines;
constexpr size_t kTwOff = kPartialsOff + kPartialsBytes;
constexpr size_t kTwBytes = 3 * kMaxN * 16;       // float4 or double2 entries
constexpr size_t kParamOff = kTwOff + kTwBytes;        // g, gamma[3]
constexpr size_t kSumsOff = kParamOff + 256;            // NQ doubles
constexpr size_t kOutOff = kSumsOff + 256;              // out6, out4
constexpr size_t kCsumOff = kOutOff + 256;              // chunk sums of the line reductions
constexpr size_t kCsumBytes = (sizeof(double) * NQ * ((kMaxLines + REDUCE_CHUNK - 1) / REDUCE_CHUNK) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCsumOff + kCsumBytes;
static_assert(kTwOff % 256 == 0 && kParamOff % 256 == 0, "scratch regions must stay aligned");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

gpe_status nfail(gpe_status s, const char *msg)
{
    set_last_error(msg);
    return s;
}

// twiddle table exp(-2 pi i t / n) evaluated in double precision: stored as
// is (complex128) or as the hi + lo float pair (complex64)
__global__ void k_noalloc_twiddles_f(float4 *tw, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    const float hx = (float)c, hy = (float)(-s);
    tw[t] = make_float4(hx, hy, (float)(c - (double)hx), (float)(-s - (double)hy));
}
__global__ void k_noalloc_twiddles_d(double2 *tw, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_double2(c, -s);
}

__global__ void k_noalloc_params(double *p, double g, double g0, double g1, double g2)
{
    p[0] = g;
    p[1] = g0;
    p[2] = g1;
    p[3] = g2;
}

int ilog2i(int64_t v)
{
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}

// Geometry of one diagnostic sweep along `axis` of a single instance.
PassArgs sweep(const gpe_plan_desc *d, const int64_t n[3], int64_t N, int axis, const void *psi, unsigned char *base,
               const double *lo, const double *h, const double *kf)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.src = psi;
    a.dst = nullptr;
    a.nax = (int)n[axis];
    a.axis = axis;
    const int64_t lpi = N / n[axis];
    a.lg_lpi = ilog2i(lpi);
    a.inst_stride = N;
    int o0, o1;
    if (axis == 0) {
        a.lg_A = 0;
        a.Sb = n[0];
        a.estride = 1;
        o0 = 1;
        o1 = 2;
    } else if (axis == 1) {
        a.lg_A = ilog2i(n[0]);
        a.Sb = n[0] * n[1];
        a.estride = n[0];
        o0 = 0;
        o1 = 2;
    } else {
        a.lg_A = ilog2i(n[0] * n[1]);
        a.Sb = N;
        a.estride = n[0] * n[1];
        o0 = 0;
        o1 = 1;
    }
    a.o0n = (int)n[o0];
    a.o1n = (int)n[o1];
    a.lg_o0 = ilog2i(n[o0]);
    a.lines_total = lpi;
    const int L = pass_lines_per_tile(d->prec, axis == 0, a.nax);
    a.ntiles = (lpi + L - 1) / L;
    a.tw = base + kTwOff + (size_t)axis * kMaxN * 16;
    a.g = reinterpret_cast<const double *>(base + kParamOff);
    a.gamma = reinterpret_cast<const double *>(base + kParamOff) + 1;
    a.partials = reinterpret_cast<double *>(base + kPartialsOff);
    a.lines_cap = kMaxLines;
    for (int i = 0; i < 3; ++i) {
        a.lo[i] = lo[i];
        a.h[i] = h[i];
        a.kf[i] = kf[i];
    }
    a.red = axis == 0 ? RED_DIAG_X : RED_DIAG_K;
    return a;
}

}  // namespace

#define NA_CUDA(call)                                                 \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return nfail(GPE_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

extern "C" gpe_status gpe_norm_energy_noalloc(const gpe_plan_desc *d, const void *psi, void *cuda_stream,
                                              double *out_host)
{
    if (!d || !psi || !out_host) return nfail(GPE_EINVAL, "gpe_norm_energy_noalloc: NULL argument");
    if (((uintptr_t)psi) % 16 != 0) return nfail(GPE_EINVAL, "psi must be 16-byte aligned");
    if (d->ndim < 1 || d->ndim > 3) return nfail(GPE_EUNSUPPORTED, "ndim must be 1, 2 or 3");
    if (d->prec != GPE_C64 && d->prec != GPE_C128) return nfail(GPE_EINVAL, "prec must be GPE_C64 or GPE_C128");
    if (d->batch != 1) return nfail(GPE_EINVAL, "gpe_norm_energy_noalloc handles one instance (batch must be 1)");
    if (d->V_host) return nfail(GPE_EUNSUPPORTED, "gpe_norm_energy_noalloc takes the harmonic trap only");
    int64_t n[3] = {1, 1, 1}, N = 1;
    double lo[3] = {0, 0, 0}, h[3] = {0, 0, 0}, kf[3] = {0, 0, 0}, dv = 1.0;
    for (int a = 0; a < d->ndim; ++a) {
        if (d->n[a] < 2 || d->n[a] > kMaxN || (d->n[a] & (d->n[a] - 1)))
            return nfail(GPE_EUNSUPPORTED, "each n[a] must be a power of two in [2, 4096]");
        if (!(d->len[a] > 0.0) || !isfinite(d->len[a]) || !isfinite(d->lo[a]) || !isfinite(d->gamma[a]))
            return nfail(GPE_EINVAL, "len[a] must be positive; lo[a] and gamma[a] finite");
        n[a] = d->n[a];
        N *= n[a];
        lo[a] = d->lo[a];
        h[a] = d->len[a] / (double)n[a];
        kf[a] = 2.0 * M_PI / d->len[a];
        dv *= h[a];
    }
    if (!isfinite(d->g)) return nfail(GPE_EINVAL, "g must be finite");
    for (int a = 0; a < d->ndim; ++a)
        if (N / n[a] > kMaxLines)
            return nfail(GPE_EUNSUPPORTED, "grid too large for the static scratch: N / n[a] must be <= "
                                           "GPE_NOALLOC_MAX_LINES (32768) on every axis");

    // the array's address on the current device, looked up on every call
    void *sym = nullptr;
    {
        cudaError_t e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
        if (e != cudaSuccess || !sym) return nfail(GPE_ECUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed");
    }
    unsigned char *base = static_cast<unsigned char *>(sym);
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // Tables and parameters of this call.  The array keeps the previous call's
    // contents: the sums and outputs are cleared; the per-line partials and the
    // twiddles are fully rewritten below before anything reads them.
    for (int a = 0; a < d->ndim; ++a) {
        const int nb = (int)((n[a] + 127) / 128);
        if (d->prec == GPE_C64)
            k_noalloc_twiddles_f<<<nb, 128, 0, st>>>(reinterpret_cast<float4 *>(base + kTwOff) + (size_t)a * kMaxN,
                                                     (int)n[a]);
        else
            k_noalloc_twiddles_d<<<nb, 128, 0, st>>>(reinterpret_cast<double2 *>(base + kTwOff) + (size_t)a * kMaxN,
                                                     (int)n[a]);
        NA_CUDA(cudaGetLastError());
    }
    k_noalloc_params<<<1, 1, 0, st>>>(reinterpret_cast<double *>(base + kParamOff), d->g,
                                      d->ndim > 0 ? d->gamma[0] : 0.0, d->ndim > 1 ? d->gamma[1] : 0.0,
                                      d->ndim > 2 ? d->gamma[2] : 0.0);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemsetAsync(base + kSumsOff, 0, 512, st));

    // the diagnostic sweeps write every per-line partial they later read
    for (int a = 0; a < d->ndim; ++a) {
        PassArgs pa = sweep(d, n, N, a, psi, base, lo, h, kf);
        NA_CUDA(launch_pass(d->prec, a == 0, pa, st));
    }
    double *partials = reinterpret_cast<double *>(base + kPartialsOff);
    double *sums = reinterpret_cast<double *>(base + kSumsOff);
    double *out6 = reinterpret_cast<double *>(base + kOutOff);
    double *out4 = out6 + 6;
    double *csum = reinterpret_cast<double *>(base + kCsumOff);
    NA_CUDA(launch_reduce_lines(partials, kMaxLines, 0, 7, 1, N / n[0], csum, sums, st));
    for (int a = 1; a < d->ndim; ++a)
        NA_CUDA(launch_reduce_lines(partials, kMaxLines, 6 + a, 1, 1, N / n[a], csum, sums, st));
    NA_CUDA(launch_finish_diag(sums, 1, d->ndim, n, dv, reinterpret_cast<const double *>(base + kParamOff), out6, out4,
                               st));
    NA_CUDA(cudaMemcpyAsync(out_host, out6, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    return GPE_OK;
}
