// resident.cu - SM-resident real-time stepping of small 2D complex64 instances.
//
// A batch of small instances (64^2 or 128^2 points, 32 or 128 KiB) does not
// need to stream through HBM at every sweep: one CTA loads an instance into
// shared memory, advances it by all steps of the call there, and writes it
// back (one read and one write of the state per call instead of two per
// step).  The CTA runs the same sequence of line transforms and pointwise
// substeps as the streaming sweeps of a 2D real-time call (prologue row sweep
// N_half.F_x; per step a column sweep F_y.K.I_y and a row sweep I_x.N.F_x,
// the last one I_x.N_half), with the same radix plan, butterflies, tables and
// pointwise code (point_op), so it gives the same bits as per-instance plans.
// CTAs loop over the batch's instances (persistent grid).
#include "pass_kernels.cuh"

namespace gpe {

template <int N> struct ResidentCfg {
    static constexpr int NT = 512;                           // threads per CTA
    static constexpr int E = 8;
    static constexpr int TPL = N / E;                        // threads per line
    static constexpr int G = NT / TPL;                       // lines transformed at once
    using Rows = GTile<float, N, 1, 1, true, E>;             // one row per thread group, swizzled exchange
    using Cols = GTile<float, N, G, 1, false, E>;            // G columns, threads across the columns
    static constexpr size_t state_bytes = sizeof(float2) * N * N;
    static constexpr size_t scr_points = (size_t)N * G;      // exchange region (rows and columns share it)
    static constexpr size_t smem = state_bytes + sizeof(float2) * scr_points + sizeof(float4) * Rows::TWN +
                                   sizeof(PassArgs) + 64;
};

template <int N>
__global__ void __launch_bounds__(ResidentCfg<N>::NT, 1) k_resident2d(const ResidentArgs ra)
{
    using Cfg = ResidentCfg<N>;
    using Rows = typename Cfg::Rows;
    using Cols = typename Cfg::Cols;
    using C = float2;
    using U = float4;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, G = Cfg::G;
    static_assert(Rows::TWN == Cols::TWN, "rows and columns share the twiddle table");
    extern __shared__ __align__(128) unsigned char smraw[];
    C *st = reinterpret_cast<C *>(smraw);
    C *scr = st + N * N;
    U *tw = reinterpret_cast<U *>(scr + Cfg::scr_points);
    PassArgs *sa = reinterpret_cast<PassArgs *>(tw + Rows::TWN);
    const int t = threadIdx.x;
    Rows::load_twiddles(tw, static_cast<const U *>(ra.tw), t, Cfg::NT);
    // row mapping: threads across the points of one row; column mapping:
    // threads across G columns
    const int rg = t / TPL, rtl = t % TPL;
    const int cl = t % G, ctl = t / G;

    for (int64_t inst = blockIdx.x; inst < ra.count; inst += gridDim.x) {
        const int ti = ra.slot_of ? ra.slot_of[inst] : (int)inst;
        C *psi = static_cast<C *>(ra.inst_ptr[inst]);
        __syncthreads();                         // the previous instance's store and args are done
        for (int i = t; i < N * N; i += Cfg::NT) st[i] = psi[i];
        if (t == 0) *sa = ra.rows;
        __syncthreads();

        // one sweep over the rows: op_pre, transform fft1, op_post (0: none)
        auto rows = [&](int op_pre, int fft1, int op_mid, int fft2) {
            for (int r0 = 0; r0 < N; r0 += G) {
                const int row = r0 + rg;
                C v[1][E];
#pragma unroll
                for (int e = 0; e < E; ++e) v[0][e] = st[row * N + rtl + TPL * e];
                point_op<float, E, TPL>(op_pre, v[0], *sa, 0, ti, row, 0, rtl, 0);
                sweep_transforms<Rows, false>(v, scr + rg * N, nullptr, rtl, 0, tw, fft1, fft2, [&]() {
                    point_op<float, E, TPL>(op_mid, v[0], *sa, 0, ti, row, 0, rtl, 0);
                });
#pragma unroll
                for (int e = 0; e < E; ++e) st[row * N + rtl + TPL * e] = v[0][e];
                __syncthreads();                 // the exchange region is reused by the next rows
            }
        };
        auto cols = [&]() {
            for (int c0 = 0; c0 < N; c0 += G) {
                const int col = c0 + cl;
                C v[1][E];
#pragma unroll
                for (int e = 0; e < E; ++e) v[0][e] = st[(ctl + TPL * e) * N + col];
                sweep_transforms<Cols, false>(v, scr, nullptr, ctl, cl, tw, -1, +1, [&]() {
                    point_op<float, E, TPL>(OP_KREAL, v[0], *sa, 0, ti, col, 0, ctl, 0);
                });
#pragma unroll
                for (int e = 0; e < E; ++e) st[(ctl + TPL * e) * N + col] = v[0][e];
                __syncthreads();
            }
        };

        // prologue: first nonlinear half-step and the forward row transform
        if (t == 0) {
            *sa = ra.rows;
            sa->vt_ax = ra.vh[0];
            sa->vt_o0 = ra.vh[1];
            sa->nl_c = 0.5 * ra.dt;
            sa->dphi = 0.0;
        }
        __syncthreads();
        rows(OP_NREAL, -1, OP_NONE, 0);
        for (int64_t s = 0; s < ra.nsteps; ++s) {
            const bool last = s == ra.nsteps - 1;
            const int d = (int)(s & (GPE_DITHER_PERIOD - 1));
            __syncthreads();
            if (t == 0) {
                *sa = ra.cols;
                if (ra.dither) {
                    sa->dither = 1;
                    for (int q = 0; q < 4; ++q) sa->dk[q] = ra.dtab[5 * d + 1 + q];
                }
            }
            __syncthreads();
            cols();
            if (t == 0) {
                *sa = ra.rows;
                sa->vt_ax = last ? ra.vh[0] : ra.vf[0];
                sa->vt_o0 = last ? ra.vh[1] : ra.vf[1];
                sa->nl_c = last ? 0.5 * ra.dt : ra.dt;
                sa->dphi = ra.dither ? ra.dtab[5 * d] : 0.0;
            }
            __syncthreads();
            rows(OP_NONE, +1, OP_NREAL, last ? 0 : -1);
        }
        __syncthreads();
        for (int i = t; i < N * N; i += Cfg::NT) psi[i] = st[i];
    }
}

template <int N> static cudaError_t launch_resident_n(const ResidentArgs &a, cudaStream_t st)
{
    using Cfg = ResidentCfg<N>;
    static LaunchCache lc;
    int cap = 0;
    cudaError_t e = prepare(k_resident2d<N>, lc, Cfg::NT, Cfg::smem, &cap);
    if (e != cudaSuccess) return e;
    if (a.count <= 0 || a.nsteps <= 0) return cudaSuccess;
    const int grid = (int)(a.count < cap ? a.count : cap);
    k_resident2d<N><<<grid, Cfg::NT, Cfg::smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resident2d(int n, const ResidentArgs &a, cudaStream_t st)
{
    if (n == 64) return launch_resident_n<64>(a, st);
    if (n == 128) return launch_resident_n<128>(a, st);
    return cudaErrorInvalidValue;
}

bool resident2d_supported(int prec, int ndim, const int64_t *n) { return prec == 0 && ndim == 2 && n[0] == n[1] && (n[0] == 64 || n[0] == 128); }

}  // namespace gpe
