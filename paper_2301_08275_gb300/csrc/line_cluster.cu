// line_cluster.cu - complex128 real-time steps of a few short lines (64, 128
// or 256 points), each line spread over a cluster of CTAs.
//
// FP64 arithmetic on this GPU issues one warp instruction per 64 cycles on
// each SM sub-partition, however many of the warp's lanes are active, so the
// time of a latency-bound step is the FP64 instruction count of the busiest
// warp.  The one-CTA-per-line kernel gives each thread 8 points of its line
// (about 700 FP64 instructions per step on one warp).  Here a line of
// N = 16 CS points is spread over a cluster of CS CTAs of one warp each, and
// each lane holds one real number: CTA c holds points CS i + c (i = 0..15),
// lane i + 16 comp the real (comp 0) or imaginary (comp 1) part of point i.
// A complex addition is then one FP64 instruction per lane and a complex
// product two; a step costs about 60.
//
// The transform is the four-step factorisation N = 16 x CS of the discrete
// Fourier transform (the split-step scheme's F and F^-1, Sec. 2 of the paper):
//   X[k1 + 16 k2] = sum_c W_CS^(c k2) W_N^(c k1) sum_i x[CS i + c] W_16^(i k1)
// Step A, the inner sums over i, is a 16-point transform within one warp
// (radix-2 stages across lanes, partners exchanged by shuffles, decimation in
// frequency: natural order in, bit-reversed out).  After the twiddle W_N^(c k1)
// the CTAs exchange their values (CTA j receives the rows k1 = j R .. j R +
// R - 1, R = 16 / CS, of every column): step B, the sums over c, is then
// again local, CS-point transforms over aligned lane groups.  The kinetic
// factor multiplies the spectrum in that layout; the inverse runs the same
// steps backwards (decimation in time: bit-reversed in, natural out) and ends
// in the layout it started from, where the nonlinear and potential factors
// of the next substep are pointwise.  Two exchanges per step, each an
// all-to-all of one 8-byte value per lane, written into the receiving CTA's
// shared memory by st.async and counted by that CTA's mbarrier.
#include <mutex>

#include "pass_kernels.cuh"

namespace gpe {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_map(unsigned a, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// write 8 bytes into CTA `rank`'s shared memory at (local address) dst and
// count them on that CTA's barrier bar
__device__ __forceinline__ void cl_send(const void *dst, const uint64_t *bar, unsigned rank, double v)
{
    const unsigned ra = cl_map(smem_addr(dst), rank);
    const unsigned rb = cl_map(smem_addr(bar), rank);
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];\n" ::"r"(ra),
                 "l"(__double_as_longlong(v)), "r"(rb)
                 : "memory");
}

__device__ __forceinline__ double flip(double v, unsigned long long sign) { return __longlong_as_double(__double_as_longlong(v) ^ sign); }

// this lane's component of (own + i other) * (wr + i wi) for lane-specific
// (a, b) = (wr, -wi) on real lanes, (wr, wi) on imaginary lanes
__device__ __forceinline__ double lane_mul(double v, double a, double b)
{
    const double o = __shfl_xor_sync(FULL, v, 16);
    return fma(v, a, o * b);
}
// v (1 + w) for an offset w given as its lane pair (a, b): small product first,
// the dominant term added last (the rounding order of the other kernels)
__device__ __forceinline__ double lane_madd1(double v, double a, double b)
{
    const double o = __shfl_xor_sync(FULL, v, 16);
    return v + fma(v, a, o * b);
}

// lane pair of the unit factor w: (wr, -wi) for comp 0, (wr, wi) for comp 1
struct Pair {
    double a, b;
};
__device__ __forceinline__ Pair pair_of(double2 w, int comp) { return {w.x, comp ? w.y : -w.y}; }
__device__ __forceinline__ Pair pair_one() { return {1.0, 0.0}; }

// W_N^m (inverse: its conjugate) from the plan's table tw[t] = exp(-2 pi i t / N)
template <int N> __device__ __forceinline__ double2 wtab(const double2 *tw, int m, bool inv)
{
    double2 w = tw[m & (N - 1)];
    if (inv) w.y = -w.y;
    return w;
}

__device__ __forceinline__ int brev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// Radix-2 stages across the lanes of aligned groups of G positions
// (position p = lane & 15, index in the group i = p & (G-1)).
// Decimation in frequency, forward: half-widths G/2 .. 1; the lower lane of a
// pair keeps the sum, the upper takes the difference times W_2H^(i mod H).
template <int G> struct LaneDft {
    static constexpr int S = G == 16 ? 4 : (G == 8 ? 3 : 2);
    Pair w[S > 1 ? S - 1 : 1];          // stage twiddles of the upper lanes (stage with H > 1)
    unsigned long long sg[S];           // sign bit of the upper lanes per stage

    template <int N> __device__ __forceinline__ void init(const double2 *tw, int p, int comp, bool inv, bool dif)
    {
        const int i = p & (G - 1);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int H = dif ? (G >> (s + 1)) : (1 << s);
            const bool up = (i & H) != 0;
            sg[s] = up ? 0x8000000000000000ull : 0ull;
            if (H > 1) {
                const int slot = dif ? s : s - 1;
                w[slot] = up ? pair_of(wtab<N>(tw, (i & (H - 1)) * (N / (2 * H)), inv), comp) : pair_one();
            }
        }
    }
    // natural order in, bit-reversed out
    __device__ __forceinline__ double dif(double v) const
    {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int H = G >> (s + 1);
            const double o = __shfl_xor_sync(FULL, v, H);
            v = flip(v, sg[s]) + o;
            if (H > 1) v = lane_mul(v, w[s].a, w[s].b);
        }
        return v;
    }
    // bit-reversed order in, natural out
    __device__ __forceinline__ double dit(double v) const
    {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int H = 1 << s;
            if (H > 1) v = lane_mul(v, w[s - 1].a, w[s - 1].b);
            const double o = __shfl_xor_sync(FULL, v, H);
            v = flip(v, sg[s]) + o;
        }
        return v;
    }
};

// Maclaurin coefficients of (cos th - 1) / th^2 and sin th / th in u = th^2,
// to u^4 (th^10 / 10! and th^9 / 9!): for |th| <= 1/16 the first omitted
// terms are below 1e-23 (cos) and 2e-21 (sin) against a factor of one
__device__ __forceinline__ void phase_coefs(int comp, double (&c)[5])
{
    if (comp == 0) {
        c[0] = -1.0 / 2.0;
        c[1] = 1.0 / 24.0;
        c[2] = -1.0 / 720.0;
        c[3] = 1.0 / 40320.0;
        c[4] = -1.0 / 3628800.0;
    } else {
        c[0] = 1.0;
        c[1] = -1.0 / 6.0;
        c[2] = 1.0 / 120.0;
        c[3] = -1.0 / 5040.0;
        c[4] = 1.0 / 362880.0;
    }
}

// v <- v exp(-i gc |v|^2), then v <- v (1 + vt) if vt is set; every lane of
// a point computes |v|^2 in the same order, so both parts turn by one angle
template <int N>
__device__ __forceinline__ double nonlinear(double v, int comp, double gc, const double (&pc)[5], bool has_v, Pair vt)
{
    const double o = __shfl_xor_sync(FULL, v, 16);
    const double re = comp ? o : v, im = comp ? v : o;
    const double th = gc * fma(re, re, im * im);
    double w;
    if (fabs(th) <= 0.0625) {
        // real lane: cos th - 1 = u P_c(u); imaginary lane: -sin th = -th P_s(u)
        const double u = th * th;
        const double pol = fma(u, fma(u, fma(u, fma(u, pc[4], pc[3]), pc[2]), pc[1]), pc[0]);
        w = (comp ? -th : u) * pol;
    } else {
        double s, c;
        sincos(0.5 * th, &s, &c);
        w = comp ? -2.0 * s * c : -2.0 * s * s;
    }
    // this lane's component of v w needs the other lane's component of w
    const double wo = __shfl_xor_sync(FULL, w, 16);
    const double wr = comp ? wo : w, wi = comp ? w : wo;
    v = v + fma(v, wr, o * (comp ? wi : -wi));
    if (has_v) v = lane_madd1(v, vt.a, vt.b);
    return v;
}

template <int CS>
__global__ void __launch_bounds__(32) k_line1d_cluster(const Line1DArgs a)
{
    constexpr int N = 16 * CS, R = 16 / CS, LGCS = CS == 16 ? 4 : (CS == 8 ? 3 : 2);
    __shared__ __align__(16) double xb[2][16][2];   // receive buffers of the two exchanges
    __shared__ __align__(8) uint64_t xbar[2];
    const int lane = threadIdx.x, p = lane & 15, comp = lane >> 4;
    const int c = (int)cl_rank();
    const int64_t inst = blockIdx.x / CS;
    double *psi = reinterpret_cast<double *>(a.inst_ptr ? a.inst_ptr[inst] : static_cast<double2 *>(a.psi) + inst * N);
    const int64_t ib = a.slot_of ? a.slot_of[inst] : inst;
    const double2 *tw = static_cast<const double2 *>(a.tw);

    if (lane == 0) {
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }

    // per-lane constants: stage twiddles, four-step twiddles, kinetic factor
    LaneDft<16> fa, ia;     // step A forward (DIF) and inverse (DIT)
    LaneDft<CS> fb, ibt;    // step B forward and inverse
    fa.template init<N>(tw, p, comp, false, true);
    ia.template init<N>(tw, p, comp, true, false);
    fb.template init<N>(tw, p, comp, false, true);
    ibt.template init<N>(tw, p, comp, true, false);
    const int k1a = brev(p, 4);                        // step A output: k1 at position p
    const Pair t4f = pair_of(wtab<N>(tw, c * k1a, false), comp);
    const int rB = p / CS, qB = p & (CS - 1);          // step B layout: position r CS + q
    const int k1b = c * R + rB;
    const Pair t4i = pair_of(wtab<N>(tw, qB * k1b, true), comp);
    Pair kin;
    {
        const int k = k1b + 16 * brev(qB, LGCS);
        double2 kt = static_cast<const double2 *>(a.kt)[k];   // exp(-i k^2 dt / 2) - 1
        kin = pair_of(make_double2((1.0 + kt.x) / N, kt.y / N), comp);
    }
    // destinations of this lane's value in the two exchanges
    const int dA = k1a / R, pA = (k1a % R) * CS + c;   // forward: CTA, position
    const int dB = qB, pB = brev(k1b, 4);              // inverse
    // potential factors at this lane's point n = CS p + c
    const int n = CS * p + c;
    const double2 *vh = static_cast<const double2 *>(a.vh), *vf = static_cast<const double2 *>(a.vf);
    const double2 *vl = a.vh_last ? static_cast<const double2 *>(a.vh_last) : vh;
    const Pair vhp = vh ? pair_of(vh[ib * N + n], comp) : pair_one();
    const Pair vfp = vf ? pair_of(vf[ib * N + n], comp) : pair_one();
    const Pair vlp = vl ? pair_of(vl[ib * N + n], comp) : pair_one();
    double pc[5];
    phase_coefs(comp, pc);
    const double g = a.g[ib];
    const double gh = g * 0.5 * a.dt, gf = g * a.dt;

    double v = psi[2 * n + comp];
    cl_sync();   // every CTA's barriers are initialised before any value is sent to it

    v = nonlinear<N>(v, comp, gh, pc, vh != nullptr, vhp);
    bool timed_out = false;
    for (int64_t st = 0; st < a.nsteps; ++st) {
        const unsigned par = (unsigned)(st & 1);
        if (lane == 0) {
            // 32 lanes x 8 bytes arrive per exchange (tx_extra: failure-handling test hook)
            mbar_expect_tx(&xbar[0], 256u + (unsigned)a.tx_extra);
            mbar_expect_tx(&xbar[1], 256u + (unsigned)a.tx_extra);
        }
        // forward transform, step A, and the exchange to the row layout
        v = fa.dif(v);
        v = lane_mul(v, t4f.a, t4f.b);
        cl_send(&xb[0][pA][comp], &xbar[0], (unsigned)dA, v);
        if (__any_sync(FULL, !mbar_wait_bounded(&xbar[0], par))) {
            timed_out = true;
            break;
        }
        v = xb[0][p][comp];
        // step B, kinetic factor (with 1/N), inverse step B
        v = fb.dif(v);
        v = lane_mul(v, kin.a, kin.b);
        v = ibt.dit(v);
        v = lane_mul(v, t4i.a, t4i.b);
        cl_send(&xb[1][pB][comp], &xbar[1], (unsigned)dB, v);
        if (__any_sync(FULL, !mbar_wait_bounded(&xbar[1], par))) {
            timed_out = true;
            break;
        }
        v = xb[1][p][comp];
        v = ia.dit(v);
        const bool last = st == a.nsteps - 1;
        v = nonlinear<N>(v, comp, last ? gh : gf, pc, (last ? vl : vf) != nullptr, last ? vlp : vfp);
    }
    if (timed_out && lane == 0 && a.err) atomicOr(a.err, (int)ERR_CLUSTER_TIMEOUT);
    // no CTA leaves while a value addressed to it can still be in flight
    cl_sync();
    psi[2 * n + comp] = v;
}

struct ClusterState {
    std::mutex mu;
    int ok[64][3] = {};    // per device and cluster size: 0 unknown, 1 usable, -1 not
};
ClusterState g_cl;

template <int CS> cudaError_t launch_cl(const Line1DArgs &a, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorNotSupported;
    const int slot = CS == 16 ? 2 : (CS == 8 ? 1 : 0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.batch * CS));
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    {
        std::lock_guard<std::mutex> lk(g_cl.mu);
        if (g_cl.ok[dev][slot] == 0) {
            if (CS > 8) cudaFuncSetAttribute(k_line1d_cluster<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            int ncl = 0;
            cudaLaunchConfig_t probe = cfg;
            probe.gridDim = dim3(CS);
            const cudaError_t oe = cudaOccupancyMaxActiveClusters(&ncl, k_line1d_cluster<CS>, &probe);
            if (oe != cudaSuccess) cudaGetLastError();
            g_cl.ok[dev][slot] = (oe == cudaSuccess && ncl >= 1) ? 1 : -1;
        }
        if (g_cl.ok[dev][slot] < 0) return cudaErrorNotSupported;
    }
    return cudaLaunchKernelEx(&cfg, k_line1d_cluster<CS>, a);
}

}  // namespace

bool line1d_cluster_applies(const Line1DArgs &a)
{
    return !a.imag && (a.n == 64 || a.n == 128 || a.n == 256) && a.batch >= 1 && a.batch <= LINE_CLUSTER_MAX_BATCH &&
           a.nsteps >= 1;
}

cudaError_t launch_line1d_cluster(const Line1DArgs &a, cudaStream_t st)
{
    switch (a.n) {
    case 64: return launch_cl<4>(a, st);
    case 128: return launch_cl<8>(a, st);
    case 256: return launch_cl<16>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe
