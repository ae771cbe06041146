// fft_tile.cuh - register/shared-memory Stockham FFT engine for tiles of lines.
//
// A CTA owns a tile of L lines of N = 2^p complex points.  Each thread holds
// E = min(8, N) points of one line in registers: point index i = tl + TPL*e
// (e = 0..E-1, TPL = N/E threads per line).  A transform is a sequence of
// Stockham passes of radix 2, 4 or 8 (the first pass takes the remainder of
// log2 N modulo 3).  In every pass the thread's butterflies read exactly the
// points it holds, so only the outputs of non-final passes go through shared
// memory; the last pass leaves point tl + TPL*e in register e again.  Two
// transforms in a row (FFT, pointwise op, IFFT) therefore need no shared-memory
// round trip between them, and loads/stores to global memory happen straight
// from registers with consecutive threads on consecutive addresses.
//
// The twiddle table holds exp(-2 pi i t / N), t < N (conjugated for inverse
// transforms).
//
// Stockham pass with radix r over sub-transforms of size Ns (Ns = product of the
// earlier radices): butterfly j (0 <= j < N/r), k = j mod Ns, reads x[j + m N/r],
// multiplies input m by W^(m k) with W = exp(dir 2 pi i / (Ns r)), takes an r-point
// DFT and writes output m to y[(j div Ns) Ns r + k + m Ns].
//
// Unit-modulus factors (twiddles, phase tables) are applied with a modulus
// error far below one ulp of the bulk precision.  A unit factor rounded to
// single precision has |w| = 1 + O(eps); applied to the same data every step,
// such errors do not average out and the norm drifts by ~1e-5 per thousand
// steps.  In single precision every table factor is therefore a pair
// hi + lo of floats (hi = fl(w), lo = fl(w - hi)) and the product v*(hi + lo)
// is formed with fused multiply-adds so that only the final value is rounded;
// the constant 1/sqrt(2) of the radix-8 butterfly is carried the same way.
// Factors whose angle is small where the data lives (kinetic and trap phases,
// the nonlinear phase) are held as offsets from one instead (cmadd1, uomul).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace gpe {

// ---------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
// complex64: both components in one packed two-lane instruction (same
// round-to-nearest result per component, half the issue slots)
template <> __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }

// Table entry of a unit factor: float -> (hi.x, hi.y, lo.x, lo.y), double -> value.
template <typename R> struct UT;
template <> struct UT<float> { using U = float4; };
template <> struct UT<double> { using U = double2; };

// v * u for a unit factor u (conj(u) when CONJ), rounding only the result
template <bool CONJ = false> __device__ __forceinline__ float2 umul(float2 v, float4 u)
{
    const float uy = CONJ ? -u.y : u.y, wy = CONJ ? -u.w : u.w;
    const float tx = fmaf(v.x, u.z, -v.y * wy);
    const float ty = fmaf(v.x, wy, v.y * u.z);
    return mk(fmaf(v.x, u.x, fmaf(-v.y, uy, tx)), fmaf(v.x, uy, fmaf(v.y, u.x, ty)));
}
template <bool CONJ = false> __device__ __forceinline__ double2 umul(double2 v, double2 u)
{
    const double uy = CONJ ? -u.y : u.y;
    return mk(fma(v.x, u.x, -v.y * uy), fma(v.x, uy, v.y * u.x));
}

// v * (1 + w) for a unit factor close to one, stored as its offset w: the
// small product v*w is formed first and v is added last, so each component is
// rounded once after the dominant term enters (rounding v*cos first and adding
// v*sin afterwards would drop the small term in a biased way).
__device__ __forceinline__ float2 cmadd1(float2 v, float2 w)
{
    return mk(v.x + fmaf(v.x, w.x, -v.y * w.y), v.y + fmaf(v.x, w.y, v.y * w.x));
}
__device__ __forceinline__ double2 cmadd1(double2 v, double2 w)
{
    return mk(v.x + fma(v.x, w.x, -v.y * w.y), v.y + fma(v.x, w.y, v.y * w.x));
}
// same with the offset held as a hi + lo float pair (table entries)
__device__ __forceinline__ float2 uomul(float2 v, float4 w)
{
    const float tx = fmaf(v.x, w.z, -v.y * w.w);
    const float ty = fmaf(v.x, w.w, v.y * w.z);
    return mk(v.x + fmaf(v.x, w.x, fmaf(-v.y, w.y, tx)), v.y + fmaf(v.x, w.y, fmaf(v.y, w.x, ty)));
}
__device__ __forceinline__ double2 uomul(double2 v, double2 w) { return cmadd1(v, w); }
// offset form of a product of two unit factors: (1+a)(1+b) - 1
template <typename C> __device__ __forceinline__ C wcomb(C a, C b)
{
    return mk(a.x + b.x + (a.x * b.x - a.y * b.y), a.y + b.y + (a.x * b.y + a.y * b.x));
}
// x / sqrt(2), with the constant carried to twice the working precision in float
__device__ __forceinline__ float mul_rsqrt2(float x)
{
    const float hi = 0.707106769084930419921875f, lo = 1.2101617e-08f;
    return fmaf(x, hi, x * lo);
}
__device__ __forceinline__ double mul_rsqrt2(double x) { return x * 0.70710678118654752440; }

// multiply by dir*i  (dir = -1: -i, dir = +1: +i)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a)
{
    if (DIR < 0) return mk(a.y, -a.x);
    return mk(-a.y, a.x);
}

// cos and sin of 2 pi j / 32 for j = 1, 2, 3 (the other non-trivial angles
// of a 32-point transform follow by symmetry), and their single-precision
// hi + lo splits: hi = fl(v), lo = fl(v - hi)
struct Trig32 {
    static constexpr double c[4] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708};
    static constexpr double s[4] = {0.0, 0.19509032201612826785, 0.38268343236508977173, 0.55557023301960222474};
};
// a * (c + i s) for constants c, s close to a unit factor; in single
// precision with hi + lo constants so that only the result is rounded
template <int J> __device__ __forceinline__ float2 cconst_mul(float2 a, bool swap_cs, float sc, float ss)
{
    constexpr float ch = (float)Trig32::c[J], cl = (float)(Trig32::c[J] - (double)(float)Trig32::c[J]);
    constexpr float sh = (float)Trig32::s[J], sl = (float)(Trig32::s[J] - (double)(float)Trig32::s[J]);
    // (c, s) or (s, c), each with a sign
    const float c_h = (swap_cs ? sh : ch) * sc, c_l = (swap_cs ? sl : cl) * sc;
    const float s_h = (swap_cs ? ch : sh) * ss, s_l = (swap_cs ? cl : sl) * ss;
    const float tx = fmaf(a.x, c_l, -a.y * s_l);
    const float ty = fmaf(a.x, s_l, a.y * c_l);
    return mk(fmaf(a.x, c_h, fmaf(-a.y, s_h, tx)), fmaf(a.x, s_h, fmaf(a.y, c_h, ty)));
}
template <int J> __device__ __forceinline__ double2 cconst_mul(double2 a, bool swap_cs, double sc, double ss)
{
    constexpr double cj = Trig32::c[J], sj = Trig32::s[J];
    const double c = (swap_cs ? sj : cj) * sc;
    const double s = (swap_cs ? cj : sj) * ss;
    return mk(fma(a.x, c, -a.y * s), fma(a.x, s, a.y * c));
}

// a * exp(DIR * 2 pi i * K / M) for M <= 32 with K a compile-time constant
// after unrolling.  Multiples of pi/2 are exact; odd multiples of pi/4 carry
// 1/sqrt(2) to twice the working precision; the other multiples of pi/16 use
// hi + lo constants (single precision), so none of these factors has a
// systematic modulus error.
template <int M, int DIR, typename C> __device__ __forceinline__ C twc(C a, int K)
{
    using R = decltype(a.x);
    const int idx = (K * (32 / M)) & 31;
    if (idx == 0) return a;
    if (idx == 8) return mul_i<DIR>(a);
    if (idx == 16) return mk(-a.x, -a.y);
    if (idx == 24) return mul_i<-DIR>(a);
    if ((idx & 7) == 4) {
        // (+-1 +- i)/sqrt(2): exp(DIR i pi idx/16) = (cx + i sy DIR)/sqrt(2)
        const R cx = (idx == 4 || idx == 28) ? (R)1 : (R)-1;
        const R sy = ((idx == 4 || idx == 12) ? (R)1 : (R)-1) * (R)DIR;
        return mk(mul_rsqrt2(cx * a.x - sy * a.y), mul_rsqrt2(sy * a.x + cx * a.y));
    }
    // angle 2 pi idx / 32 = q pi/2 + j pi/16 with j in 1..3 (first quadrant
    // reference angle j or 8 - j)
    const int q = idx >> 3, j = idx & 7;          // j in {1,2,3,5,6,7}
    const bool sw = j > 4;                         // reference angle (8 - j): swap cos and sin
    const int jj = sw ? 8 - j : j;
    // cos and sin of the angle in quadrant q: signs and swap
    //   q=0: ( c,  s); q=1: (-s,  c); q=2: (-c, -s); q=3: ( s, -c)
    // with (c, s) = (cos, sin)(jj pi/16) or swapped when sw
    const bool qs = (q & 1) != 0;
    const bool swap_cs = sw != qs;
    const R sgn_c = (q == 1 || q == 2) ? (R)-1 : (R)1;
    const R sgn_s = ((q >= 2) ? (R)-1 : (R)1) * (R)DIR;
    if (jj == 1) return cconst_mul<1>(a, swap_cs, sgn_c, sgn_s);
    if (jj == 2) return cconst_mul<2>(a, swap_cs, sgn_c, sgn_s);
    return cconst_mul<3>(a, swap_cs, sgn_c, sgn_s);
}

// one radix-2 step of the M-point DFT: lo = e + W^k o, hi = e - W^k o with
// W = exp(DIR 2 pi i / M).  The factors 1, -1 and +-i are folded into the
// additions (no negated or swapped operand is formed); the others multiply
// first and add with packed instructions.
template <int M, int DIR, typename C> __device__ __forceinline__ void bfly(C e, C o, int k, C &lo, C &hi)
{
    const int idx = (k * (32 / M)) & 31;
    if (idx == 0) {
        lo = cadd(e, o);
        hi = csub(e, o);
    } else if (idx == 16) {
        lo = csub(e, o);
        hi = cadd(e, o);
    } else if (idx == 8 || idx == 24) {
        // W^k = s i, s = +-1: e + s i o = (e.x - s o.y, e.y + s o.x)
        const bool plus = (idx == 8) == (DIR > 0);
        if (plus) {
            lo = mk(e.x - o.y, e.y + o.x);
            hi = mk(e.x + o.y, e.y - o.x);
        } else {
            lo = mk(e.x + o.y, e.y - o.x);
            hi = mk(e.x - o.y, e.y + o.x);
        }
    } else {
        const C t = twc<M, DIR>(o, k);
        lo = cadd(e, t);
        hi = csub(e, t);
    }
}

// In-register DFT of size M (1, 2, 4, 8, 16, 32): even/odd split (radix-2 DIT),
// natural-order input and output.  DIR = -1 forward, +1 inverse.
template <int M, int DIR, typename C> struct Dft {
    __device__ __forceinline__ static void run(C *x)
    {
        C e[M / 2], o[M / 2];
#pragma unroll
        for (int i = 0; i < M / 2; ++i) { e[i] = x[2 * i]; o[i] = x[2 * i + 1]; }
        Dft<M / 2, DIR, C>::run(e);
        Dft<M / 2, DIR, C>::run(o);
#pragma unroll
        for (int k = 0; k < M / 2; ++k) bfly<M, DIR>(e[k], o[k], k, x[k], x[k + M / 2]);
    }
};
template <int DIR, typename C> struct Dft<1, DIR, C> {
    __device__ __forceinline__ static void run(C *) {}
};
template <int DIR, typename C> struct Dft<2, DIR, C> {
    __device__ __forceinline__ static void run(C *x)
    {
        C a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

// ---------------------------------------------------------------- pass plan
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

template <int N> struct Radix {
    static constexpr int LG = ilog2c(N);
    static constexpr int E = N >= 8 ? 8 : N;           // points per thread
    static constexpr int REM = N >= 8 ? LG % 3 : 0;    // log2 of the first pass when not 8
    static constexpr int P = N < 8 ? 1 : LG / 3 + (REM ? 1 : 0);
    __host__ __device__ static constexpr int radix(int p) { return N < 8 ? N : ((REM && p == 0) ? (1 << REM) : 8); }
    __host__ __device__ static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
};
// Pass plan for threads holding 32 points of a line (N >= 32): a radix-32
// first pass (no twiddles), then the remaining log2(N/32) bits in passes of
// at most 32: 256 = 32 x 8, 512 = 32 x 16, 1024 = 32 x 32, 2048 = 32 x 8 x 8,
// 4096 = 32 x 16 x 8.  Each transform then needs one shared-memory exchange
// per pass after the first (one for 256..1024 points, against two with
// radix-8 passes).
template <int N> struct Radix32 {
    static constexpr int LG = ilog2c(N);
    static constexpr int E = 32;
    static constexpr int REST = LG - 5;
    static constexpr int P = REST <= 0 ? 1 : (REST <= 5 ? 2 : 3);
    __host__ __device__ static constexpr int radix(int p)
    {
        return p == 0 ? (N < 32 ? N : 32)
                      : (P == 2 ? (1 << REST) : (p == 1 ? (1 << (REST - REST / 2)) : (1 << (REST / 2))));
    }
    __host__ __device__ static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
};
template <int N, int E> struct PassPlan { using T = Radix<N>; };
template <int N> struct PassPlan<N, 32> { using T = Radix32<N>; };

// ---------------------------------------------------------------- tile engine
// ROWS = true : lines are contiguous rows (x axis); shared layout row-major with
//               the point index XOR-swizzled inside each 128-byte block
//               (i ^ ((i / P) mod P), P points per 128 bytes), which keeps both
//               the contiguous reads and the stride-r Stockham writes free of
//               bank conflicts.
// ROWS = false: lines are strided (y or z axis); L lines interleaved point by point.
template <typename R, int N, int L, bool ROWS> struct Tile {
    using C = typename CT<R>::C;
    static constexpr int E = Radix<N>::E;
    static constexpr int TPL = N / E;
    static constexpr int NT = L * TPL;
    static constexpr int P = 128 / (int)sizeof(C);      // points per 128-byte block
    static constexpr int SMEM_POINTS = N * L;

    __device__ __forceinline__ static int sidx(int i, int l)
    {
        if (ROWS) return l * N + (i ^ ((i / P) & (P - 1)));
        return i * L + l;
    }
    __device__ __forceinline__ static int line_of(int t) { return ROWS ? t / TPL : t % L; }
    __device__ __forceinline__ static int tl_of(int t) { return ROWS ? t % TPL : t / L; }

    using U = typename UT<R>::U;

    // One pass p of the transform.  v holds points tl + TPL*e.
    template <int DIR, int p>
    __device__ __forceinline__ static void pass(C (&v)[E], C *sm, int tl, int l, const U *__restrict__ tw)
    {
        constexpr int r = Radix<N>::radix(p);
        constexpr int Ns = Radix<N>::ns(p);
        constexpr int B = E / r;
        constexpr bool last = (p == Radix<N>::P - 1);
        if constexpr (p > 0) {
            __syncthreads();                          // previous pass outputs visible
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sm[sidx(tl + TPL * e, l)];
            if constexpr (!last) __syncthreads();     // all reads done before rewriting
        } else if constexpr (!last) {
            __syncthreads();                          // earlier readers of sm are done
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const int j = tl + q * TPL;
            const int k = j & (Ns - 1);
            C x[r];
#pragma unroll
            for (int m = 0; m < r; ++m) x[m] = v[q + m * B];
            if constexpr (Ns > 1) {
#pragma unroll
                for (int m = 1; m < r; ++m) x[m] = umul<(DIR > 0)>(x[m], tw[m * k * (N / (Ns * r))]);
            }
            Dft<r, DIR, C>::run(x);
            if constexpr (last) {
#pragma unroll
                for (int m = 0; m < r; ++m) v[q + m * B] = x[m];
            } else {
                const int base = (j / Ns) * Ns * r + k;
#pragma unroll
                for (int m = 0; m < r; ++m) sm[sidx(base + m * Ns, l)] = x[m];
            }
        }
    }

    // Full N-point transform of the thread's line, in place in registers.
    // DIR = -1 forward (unnormalised), +1 inverse (unnormalised).
    template <int DIR, int p = 0>
    __device__ __forceinline__ static void fft(C (&v)[E], C *sm, int tl, int l, const U *tw)
    {
        if constexpr (p < Radix<N>::P) {
            pass<DIR, p>(v, sm, tl, l, tw);
            fft<DIR, p + 1>(v, sm, tl, l, tw);
        }
    }
};

// ---------------------------------------------------------------- line groups
// Strided tile in which each thread carries LPT adjacent lines: the points
// (i, l0) ... (i, l0+LPT-1) are adjacent in shared memory and one twiddle read
// serves all of them.  Thread t works on lines l0 = LPT*(t % NP) ... and
// points tl + TPL*e with tl = t / NP.
//
// SW = true XOR-swizzles the point index: the low bits of i are flipped by the
// bits just above the first radix, so that the stride-r writes of the first
// Stockham pass (lanes with consecutive tl write points r apart) fall into
// distinct 128-byte bank rows when a point row (L points) is narrower than a
// bank row.  The map is a bijection of [0, N): every flipped bit is flipped by
// a higher bit, which it does not change.
//
// EPT points per thread (0: Radix<N>::E = 8): with 16, each pass runs two
// butterflies per thread (more independent work per thread, half the threads
// per line); the arithmetic of every butterfly is the same.  With 32 the
// passes follow Radix32 (a radix-32 first pass, one exchange fewer per
// transform for 256 to 1024 points).
//
// PAD = true (without SW) inserts one point row (L points) after every PB
// points, PB the first pass's radix, where a row is narrower than a bank row:
// point i of line l sits at (i + i/PB)*L + l.  The first pass's writes, PB
// points apart in lanes with consecutive tl, then land one row apart instead
// of on the same banks (the 8-line tile of 512 points: 4 wavefronts per
// warp store -> 2).  The pad is free: in every access pattern of the passes
// the point index splits into a per-thread part and a constant with disjoint
// bits, and i/PB splits with it (no carry), so the pad folds into the
// thread's base and the constant offsets (layout_consistent checks this).
template <typename R, int N, int L, int LPT, bool SW = false, int EPT = 0, bool PAD = false> struct GTile {
    using C = typename CT<R>::C;
    using U = typename UT<R>::U;
    static constexpr int E = EPT ? EPT : Radix<N>::E;
    using PL = typename PassPlan<N, E>::T;      // radix of each pass
    static_assert(E >= PL::radix(0) && N % E == 0, "points per thread must cover the largest radix");
    static constexpr int TPL = N / E;
    static constexpr int LPT_ = LPT;
    static constexpr int NP = L / LPT;
    static constexpr int NT = NP * TPL;
    static constexpr int SMEM_POINTS = N * L;
    static_assert(L % LPT == 0, "lines per tile must be a multiple of lines per thread");

    static constexpr int QS = 128 / (L * (int)sizeof(C)) > 1 ? 128 / (L * (int)sizeof(C)) : 1;
    static constexpr int SWS = ilog2c(PL::radix(0));
    static constexpr int PB = PL::radix(0);
    static constexpr bool PADDED = PAD && !SW && QS > 1 && PL::P > 1;
    // points of one tile buffer (the padded layout takes N/PB rows more),
    // a whole number of KiB so that consecutive buffers stay aligned
    static constexpr int BUF_POINTS =
        PADDED ? (((N + N / PB) * L * (int)sizeof(C) + 1023) / 1024) * (1024 / (int)sizeof(C)) : SMEM_POINTS;
    __host__ __device__ __forceinline__ static constexpr int sidx(int i, int l)
    {
        if constexpr (SW) return (i ^ ((i >> SWS) & (QS - 1))) * L + l;
        if constexpr (PADDED) return (i + i / PB) * L + l;
        return i * L + l;
    }

    // index of a thread's own point tl + TPL*e.  When TPL is a multiple of QS
    // and of the first radix, the swizzle key of i depends on tl and on e only
    // through a constant, and XOR-ing it leaves TPL*e untouched: the index is
    // (tl ^ key) + TPL*e, a per-thread base plus a constant (same value as sidx).
    __host__ __device__ __forceinline__ static constexpr int sidx_own(int tl, int e, int l)
    {
        if constexpr (PADDED && PB % TPL == 0) {
            // tl < TPL and TPL*e mod PB is a multiple of TPL below PB
            return (tl + TPL * e + (TPL * e) / PB) * L + l;
        } else if constexpr (SW && TPL % QS == 0 && TPL % (1 << SWS) == 0) {
            const int key = ((tl >> SWS) + (TPL >> SWS) * e) & (QS - 1);
            return ((tl ^ key) + TPL * e) * L + l;
        } else {
            return sidx(tl + TPL * e, l);
        }
    }

    __device__ __forceinline__ static void ld(const C *sm, int tl, int e, int l0, C (&v)[LPT][E])
    {
        const int i0 = sidx_own(tl, e, l0);
        if constexpr (LPT == 2 && sizeof(C) == 8) {
            const float4 q = *reinterpret_cast<const float4 *>(sm + i0);
            v[0][e] = mk(q.x, q.y);
            v[1][e] = mk(q.z, q.w);
        } else {
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) v[ln][e] = sm[i0 + ln];
        }
    }
    // the same without the swizzle (point i of line l at i*L + l)
    __device__ __forceinline__ static void ld_plain(const C *sm, int tl, int e, int l0, C (&v)[LPT][E])
    {
        const int i0 = (tl + TPL * e) * L + l0;
#pragma unroll
        for (int ln = 0; ln < LPT; ++ln) v[ln][e] = sm[i0 + ln];
    }
    // swizzled point index before the line interleave
    __host__ __device__ static constexpr int sraw(int i) { return SW ? (i ^ ((i >> SWS) & (QS - 1))) : i; }
    // Index of Stockham output base + m*Ns of a pass.  base and m*Ns occupy
    // disjoint bits (base = (j div Ns) Ns r + k with k < Ns, m < r), so do their
    // shifted copies, and the swizzle is linear over XOR on such pairs:
    // sraw(base + m Ns) = sraw(base) ^ sraw(m Ns), the second a constant.
    template <int Ns> __host__ __device__ __forceinline__ static constexpr int sidx_out(int sb, int m, int l)
    {
        if constexpr (SW) return (sb ^ sraw(m * Ns)) * L + l;
        if constexpr (PADDED) return (sb + m * Ns + (m * Ns) / PB) * L + l;
        return (sb + m * Ns) * L + l;
    }
    // the per-thread part of sidx_out (base without the line interleave)
    __host__ __device__ __forceinline__ static constexpr int sbase(int base)
    {
        return SW ? sraw(base) : PADDED ? base + base / PB : base;
    }
    // every access pattern of the passes addresses point i of line l at
    // sidx(i, l), and the largest index fits a tile buffer
    template <int p = 0> static constexpr bool out_consistent()
    {
        if constexpr (p + 1 >= PL::P) {
            return true;      // the last pass keeps its results in registers
        } else {
            constexpr int r = PL::radix(p), Ns = PL::ns(p), B = E / r;
            for (int tl = 0; tl < TPL; ++tl)
                for (int q = 0; q < B; ++q) {
                    const int j = tl + q * TPL, k = j & (Ns - 1);
                    const int base = (j / Ns) * Ns * r + k;
                    for (int m = 0; m < r; ++m)
                        if (sidx_out<Ns>(sbase(base), m, 0) != sidx(base + m * Ns, 0)) return false;
                }
            return out_consistent<p + 1>();
        }
    }
    static constexpr bool layout_consistent()
    {
        for (int tl = 0; tl < TPL; ++tl)
            for (int e = 0; e < E; ++e)
                if (sidx_own(tl, e, 0) != sidx(tl + TPL * e, 0)) return false;
        int mx = 0;
        for (int i = 0; i < N; ++i) mx = sidx(i, L - 1) > mx ? sidx(i, L - 1) : mx;
        return mx < BUF_POINTS && out_consistent<0>();
    }
    __device__ __forceinline__ static void st_at(C *sm, int i0, const C *x)
    {
        if constexpr (LPT == 2 && sizeof(C) == 8) {
            *reinterpret_cast<float4 *>(sm + i0) = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
        } else {
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) sm[i0 + ln] = x[ln];
        }
    }

    // Twiddles in shared memory are laid out pass by pass: pass p (Ns > 1)
    // owns (r-1)*Ns entries at tw_off(p), entry (m-1)*Ns + k = W_{Ns r}^(m k).
    // Lanes with consecutive k then read consecutive 16-byte entries (no bank
    // conflicts) and each thread's r-1 reads sit at constant offsets.
    __host__ __device__ static constexpr int tw_off(int p)
    {
        return p <= 1 ? 0 : tw_off(p - 1) + PL::ns(p - 1) * (PL::radix(p - 1) - 1);
    }
    static constexpr int TWN = tw_off(PL::P);
    // fill the pass-ordered table from the natural one (W_N^t, t < N)
    __device__ __forceinline__ static void load_twiddles(U *tws, const U *__restrict__ twg, int t, int nt)
    {
        for (int idx = t; idx < TWN; idx += nt) tws[idx] = twg[tw_src<1>(idx)];
    }
    template <int p> __device__ __forceinline__ static int tw_src(int idx)
    {
        if constexpr (p >= PL::P) {
            return 0;
        } else {
            constexpr int ns = PL::ns(p), r = PL::radix(p);
            const int rel = idx - tw_off(p);
            if (rel < ns * (r - 1)) {
                const int m = rel / ns + 1, k = rel % ns;
                return m * k * (N / (ns * r));
            }
            return tw_src<p + 1>(idx);
        }
    }

    // Shared-memory regions of the passes.  Without PING every non-final pass
    // writes the tile buffer sb, after a barrier that follows all reads of the
    // previous pass (two barriers per pass).  With PING the outputs alternate
    // between a scratch region ss (even passes) and sb (odd passes): the region
    // a pass writes was last read one pass earlier, before the barrier that
    // opens the pass, so one barrier per pass suffices.  Pass 0 then needs none
    // when the pass count is odd: the previous transform (or tile) last read ss
    // in a pass that a later barrier closed.  A transform's input registers
    // must not depend on pending reads of ss or sb by other threads beyond
    // these rules (the tile's own load from sb is closed by the barrier of pass 1).
    template <int DIR, int p, bool PING = false>
    __device__ __forceinline__ static void pass(C (&v)[LPT][E], C *sb, C *ss, int tl, int l0,
                                                const U *__restrict__ tw)
    {
        constexpr int r = PL::radix(p);
        constexpr int Ns = PL::ns(p);
        constexpr int B = E / r;
        constexpr bool last = (p == PL::P - 1);
        C *const rd = (PING && p % 2 == 1) ? ss : sb;    // written by pass p-1
        C *const wr = (PING && p % 2 == 0) ? ss : sb;
        if constexpr (p > 0) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) ld(rd, tl, e, l0, v);
            if constexpr (!last && !PING) __syncthreads();
        } else if constexpr (!last && (!PING || PL::P % 2 == 0)) {
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const int j = tl + q * TPL;
            const int k = j & (Ns - 1);
            C x[LPT][r];
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln)
#pragma unroll
                for (int m = 0; m < r; ++m) x[ln][m] = v[ln][q + m * B];
            if constexpr (Ns > 1) {
                const U *twk = tw + tw_off(p) + k;
#pragma unroll
                for (int m = 1; m < r; ++m) {
                    const U w = twk[(m - 1) * Ns];
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln) x[ln][m] = umul<(DIR > 0)>(x[ln][m], w);
                }
            }
#pragma unroll
            for (int ln = 0; ln < LPT; ++ln) Dft<r, DIR, C>::run(x[ln]);
            if constexpr (last) {
#pragma unroll
                for (int ln = 0; ln < LPT; ++ln)
#pragma unroll
                    for (int m = 0; m < r; ++m) v[ln][q + m * B] = x[ln][m];
            } else {
                const int base = (j / Ns) * Ns * r + k;
                const int sb = sbase(base);
#pragma unroll
                for (int m = 0; m < r; ++m) {
                    C y[LPT];
#pragma unroll
                    for (int ln = 0; ln < LPT; ++ln) y[ln] = x[ln][m];
                    st_at(wr, sidx_out<Ns>(sb, m, l0), y);
                }
            }
        }
    }

    template <int DIR, bool PING = false, int p = 0>
    __device__ __forceinline__ static void fft(C (&v)[LPT][E], C *sb, C *ss, int tl, int l0, const U *tw)
    {
        if constexpr (p < PL::P) {
            pass<DIR, p, PING>(v, sb, ss, tl, l0, tw);
            fft<DIR, PING, p + 1>(v, sb, ss, tl, l0, tw);
        }
    }

    // v <- conj(v) (exact).  Sweeps that run a forward and an inverse
    // transform compute the inverse as conj(F(conj(v))) inside a two-iteration
    // loop around one copy of the forward code (see sweep_transforms): half
    // the instruction footprint, which matters where a CTA runs its code only
    // once or twice per launch (grids of a few thousand lines).
    __device__ __forceinline__ static void conj(C (&v)[LPT][E])
    {
#pragma unroll
        for (int ln = 0; ln < LPT; ++ln)
#pragma unroll
            for (int e = 0; e < E; ++e) v[ln][e].y = -v[ln][e].y;
    }
};

// Two transforms with a pointwise step between them, f1, f2 in {-1 forward,
// +1 inverse, 0 none}: one copy of the forward transform in a loop, the
// inverse as conj(F(conj(v))).  Every kernel of the library that runs the
// 2D/3D sweeps goes through here, so all of them round alike.
template <typename T, bool PING, typename Mid>
__device__ __forceinline__ void sweep_transforms(typename T::C (&v)[T::LPT_][T::E], typename T::C *sb,
                                                 typename T::C *ss, int tl, int l0, const typename T::U *tw, int f1,
                                                 int f2, Mid &&mid)
{
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int f = h ? f2 : f1;
        if (f != 0) {
            if (f > 0) T::conj(v);
            T::template fft<-1, PING>(v, sb, ss, tl, l0, tw);
            if (f > 0) T::conj(v);
        }
        if (h == 0) mid();
    }
}

}  // namespace gpe
