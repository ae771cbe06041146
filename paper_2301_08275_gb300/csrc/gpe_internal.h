// gpe_internal.h - launch descriptors shared by the library's translation units.
#pragma once
#include <cuda.h>            // CUtensorMap (type only; the driver entry point is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpe {

// pointwise operations a pass applies to every point it holds
enum PointOp : int {
    OP_NONE = 0,
    OP_NREAL = 1,        // psi *= Vphase(x) exp(-i g c |psi|^2)        (real-time nonlinear substep)
    OP_NIMAG = 2,        // psi *= Vdecay(x) exp(-g c |psi|^2)          (imaginary-time nonlinear substep)
    OP_KREAL = 3,        // psi *= prod_a exp(-i k_a^2 dt/2)/n_a          (real-time kinetic substep)
    OP_KIMAG = 4,        // psi *= prod_a exp(-k_a^2 dt/2)/n_a            (imaginary-time kinetic substep)
    OP_SCALE_NIMAG = 5,  // psi *= s[instance], then OP_NIMAG            (deferred renormalisation)
    OP_SCALE = 6,        // psi *= s[instance]
};

// reductions a pass can produce, one value per line per quantity
enum PassReduce : int {
    RED_NONE = 0,
    RED_NORM = 1,    // q0 = sum |psi|^2 of the final point values
    RED_DIAG_X = 2,  // x rows: q0 sum rho, q1 sum x^2 rho, q2 sum y^2 rho, q3 sum z^2 rho,
                     //         q4 sum V rho, q5 sum rho^2, q6 sum kx^2 |F_x psi|^2 (no store)
    RED_DIAG_K = 3,  // y or z lines: q(6+axis) sum k^2 |F_axis psi|^2 (no store)
    RED_DIAG_XM = 4, // x rows: the real-space moments of RED_DIAG_X only (q6 = 0, no transform)
};

enum { NQ = 9 };     // reduction quantities per line

struct PassArgs {
    const void *src;
    void *dst;
    int64_t ntiles;        // tiles of L lines
    int64_t lines_total;   // batch * lines per instance
    int lg_lpi;            // log2(lines per instance)
    int lg_A;              // line li starts at (li & (A-1)) + (li >> lg_A) * Sb
    int64_t Sb;
    int64_t estride;       // element stride along the line
    int64_t inst_stride;   // elements between instances
    int lg_o0;             // other-axis coordinates: c0 = li & (o0n-1), c1 = li >> lg_o0
    int o0n, o1n;          // sizes of the other axes (1 if absent)
    int nax;               // points on this axis
    int axis;              // 0, 1, 2
    int op_pre, fft1, op_mid, fft2, op_post, red;   // fft: 0 none, -1 forward, +1 inverse
    // unit-factor tables: double2 values (complex128) or float4 hi/lo pairs (complex64)
    const void *tw;        // exp(-2 pi i t / nax), t < nax
    // trap tables per instance ([batch][n]); NULL when the trap is off on that axis
    const void *vt_ax, *vt_o0, *vt_o1;   // offsets exp(-i V_a c) - 1
    const void *vi_ax, *vi_o0, *vi_o1;   // real    exp(-V_a c)
    // kinetic tables ([n]); NULL when absent (1D/2D other axes)
    const void *kt_ax, *kt_o0, *kt_o1;   // offsets exp(-i k_a^2 dt/2) - 1
    const void *ki_ax, *ki_o0, *ki_o1;   // real
    // potential sampled at the grid points ([N] of one instance, shared by all;
    // real type of the bulk precision), or NULL: vsamp enters the nonlinear
    // substeps, vsamp_diag the potential energy (both set for 2D/3D; 1D steps
    // take the same values through the trap tables, so only vsamp_diag is set)
    const void *vsamp, *vsamp_diag;
    const double *g;       // per-instance interaction
    double nl_c;           // theta = g * nl_c * |psi|^2
    // per-step phase dither of the complex64 real-time step: the kinetic
    // substep multiplies by exp(-i phi) as well (dk: its offset exp(-i phi) - 1
    // as a hi, hi, lo, lo float quadruple stored in doubles) and the following
    // nonlinear substep by exp(+i phi) (dphi = phi); 0 when off
    int dither;
    double dk[4];
    double dphi;
    double inv_n;          // 1/N applied with the kinetic substep
    // programmatic dependent launch: 1 lets the next kernel of the stream
    // start its launch as soon as every CTA of this one has begun (grids that
    // are resident at once: small states), 0 once every CTA has written its
    // tiles (so that waiting CTAs of the next kernel do not hold SM resources
    // while this one still has tiles to run)
    int pdl_early;
    // device-side stop of an imaginary-time run: when set and *stop != 0 at
    // launch, the kernel leaves without touching anything
    const int *stop;
    const double *scale;   // per-instance renormalisation factor
    // optional indirection for batches of separately allocated instances:
    // instance b lives at inst_ptr[b] (src = dst = that pointer) and takes its
    // parameters and trap tables from slot slot_of[b] instead of b
    void *const *inst_ptr;
    const int *slot_of;
    double *partials;      // [NQ][lines_cap] per-line sums
    int64_t lines_cap;
    int64_t line0;         // first line of the sweep (a slab of the grid): lines line0 .. lines_total - 1
    // diagnostics geometry
    const double *gamma;   // [batch][3]
    double lo[3], h[3], kf[3];   // box corner, spacing, 2 pi / len per axis
    // tile staging by the tensor-memory accelerator (strided axes only): when
    // tma_chunks > 0 each tile is fetched as tma_chunks boxes of tma_box points
    // along the axis through the tensor map passed beside these arguments
    int tma_chunks, tma_box;
    int tx_extra;          // bytes added to each tile's expected count (0; > 0 only in the
                           // failure-handling test, so that the wait runs out)
    int *err;              // device error word (bit ERR_TMA_TIMEOUT), may be NULL
    int generic;           // host side: 1 launches the generic kernel whatever the program
};

enum : int {
    ERR_NUMERIC = 1,       // non-finite or zero norm in a renormalisation
    ERR_TMA_TIMEOUT = 2,   // a tile copy did not complete within the wait limit
    ERR_CLUSTER_TIMEOUT = 4,   // a cluster exchange did not complete within the wait limit
};

// record the thread-local message returned by gpe_last_error()
void set_last_error(const char *msg);

// launch one pass; returns cudaSuccess or the launch error
// tmap: tensor map of the swept array when a.tma_chunks > 0, else NULL;
// var: tile shape (0 or 1, see pass_kernels.cuh)
cudaError_t launch_pass(int prec, bool rows, const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap = nullptr,
                        int var = 0);
int pass_lines_per_tile(int prec, bool rows, int n, int var = 0);

// whole 1D steps with each line (instance) resident on chip for all steps
// Real-time stepping of small 2D complex64 instances held in shared memory
// for a whole call (resident.cu).
#define GPE_DITHER_PERIOD 65536   // the phase dither sequence repeats after this many steps
struct ResidentArgs {
    void *const *inst_ptr;     // instance b at inst_ptr[b] (n x n points, x fastest)
    const int *slot_of;        // its parameter/table slot, or NULL (slot b)
    int64_t count, nsteps;
    const void *tw;            // natural twiddle table of the n-point lines
    PassArgs rows, cols;       // argument templates of the row (nonlinear) and column (kinetic) sweeps
    const void *vh[2], *vf[2]; // trap tables of x and y (half and full steps), or NULL
    double dt;
    int dither;                // 1: the complex64 phase dither of the real-time step
    const double *dtab;        // [GPE_DITHER_PERIOD][5]: phi, then the offset of exp(-i phi) as hi, hi, lo, lo
};
cudaError_t launch_resident2d(int n, const ResidentArgs &a, cudaStream_t st);
bool resident2d_supported(int prec, int ndim, const int64_t *n);

struct Line1DArgs {
    void *psi;
    int64_t batch;
    int n;
    int64_t nsteps;
    int imag;               // 0 real time, 1 imaginary time with per-step renormalisation
    const void *tw;
    const void *kt;         // offsets exp(-i k^2 dt/2) - 1 (real time) or exp(-k^2 dt/2)/n (imag)
    const void *vh, *vf;    // offsets exp(-i V dt/2) - 1, exp(-i V dt) - 1 ([batch][n]) or NULL
    const void *vh_last;    // optional: the last half-step's table instead of vh (time-dependent trap)
    const void *vi;         // real decay table (imag) or NULL
    const double *g;
    double dt;
    double target_norm_over_dv;   // imag: target norm / cell volume
    int *err;               // set to 1 if a norm turns non-finite or zero
    void *const *inst_ptr;  // optional: instance b lives at inst_ptr[b]
    const int *slot_of;     // optional: parameter/table slot of instance b
    int cluster;            // 1: complex128 real-time steps may take the cluster kernel
    int tx_extra;           // test hook: bytes each cluster exchange waits for beyond what arrives
    const int *stop;        // as PassArgs::stop
};
cudaError_t launch_line1d(int prec, const Line1DArgs &a, cudaStream_t st);
// complex128 real-time steps of at most LINE_CLUSTER_MAX_BATCH lines of 64,
// 128 or 256 points, one line per cluster of 4, 8 or 16 CTAs (line_cluster.cu);
// cudaErrorNotSupported when the device cannot place such a cluster
constexpr int64_t LINE_CLUSTER_MAX_BATCH = 32;
bool line1d_cluster_applies(const Line1DArgs &a);
cudaError_t launch_line1d_cluster(const Line1DArgs &a, cudaStream_t st);

// trap tables of one time level of a time-dependent harmonic trap (diag_spec.cu):
// for every axis a < ndim and every instance, tab[a][b*n[a] + j] = exp(-i V_a c) - 1
// with V_a = gamma[a]^2 x_j^2 / 2, x_j = lo[a] + j h[a] (float4 hi/lo pairs for
// prec 0, double2 for prec 1)
cudaError_t launch_trap_level(int prec, void *const *tab, int ndim, const int64_t *n, const double *lo,
                              const double *h, const double *gamma, double c, int64_t batch, cudaStream_t st);

// reductions and spectra (diag_spec.cu)
// sums[b*NQ + q], q in [nq_first, nq_first + nq): per-instance sums of the
// per-line partials, in a fixed order (chunks of REDUCE_CHUNK lines, then the
// chunk sums); csum is scratch of batch * NQ * reduce_chunks(lines_per_inst)
// doubles.  With scale set, the q = 0 sum also gives the renormalisation
// factor scale[b] = sqrt(target / (sum * dv)) (err |= ERR_NUMERIC and
// scale[b] = 1 for a zero or non-finite norm).
constexpr int64_t REDUCE_CHUNK = 4096;
int64_t reduce_chunks(int64_t lines_per_inst);
cudaError_t launch_reduce_lines(const double *partials, int64_t lines_cap, int nq_first, int nq, int64_t batch,
                                int64_t lines_per_inst, double *csum, double *sums, cudaStream_t st,
                                double dv = 0.0, double target = 0.0, double *scale = nullptr, int *err = nullptr,
                                const int *stop = nullptr);
cudaError_t launch_finish_diag(const double *sums, int64_t batch, int ndim, const int64_t *n, double dv,
                               const double *g, double *out6, double *out4, cudaStream_t st,
                               const int *stop = nullptr);
// Device-side convergence test of gpe_step_imag: imag_init takes the energies
// of out6 as the first reference and clears the stop word and step counter;
// imag_check (after each chunk of `chunk` steps and its diagnostics), unless
// *stop is already set, adds chunk to *done, compares every instance's energy
// with its reference (|E - E_prev| < etol for all: *stop = 1; a non-finite
// energy or a set ERR_NUMERIC bit in *err: *stop = 2) and makes it the new
// reference.  The kernels of later chunks see *stop and do nothing.
cudaError_t launch_imag_init(const double *out6, double *eprev, int64_t batch, int *stop, int64_t *done,
                             cudaStream_t st);
cudaError_t launch_imag_check(const double *out6, double *eprev, int64_t batch, double etol, int64_t chunk, int *stop,
                              int64_t *done, const int *err, cudaStream_t st);

struct SpecArgs {
    int prec;
    int ndim;
    int64_t n[3];
    double kf[3];       // 2 pi / len
    double lratio[3];   // max_len / len
    int64_t N;
    int part;           // k_velocity: 0 u = Im(conj(psi) d psi)/|psi|, 1 w = Re(...)/|psi| = d|psi|
    int split;          // k_bin: 1 incompressible / compressible parts, 0 total of the components
    int ncomp;          // k_bin: field components summed (ndim, or 1 for psi_hat itself)
};
cudaError_t launch_deriv(const SpecArgs &s, const void *src, void *dst, int axis, cudaStream_t st);
cudaError_t launch_velocity(const SpecArgs &s, const void *psi, void *w, cudaStream_t st);
cudaError_t launch_bin(const SpecArgs &s, void *const *uh, int64_t nshells, double *block_hist, int nblocks,
                       double *aux, cudaStream_t st);
cudaError_t launch_hist_reduce(const double *block_hist, int nblocks, int64_t nshells, double dv_over_n,
                               const double *aux, double *out_inc, double *out_comp, cudaStream_t st);
int bin_blocks(const SpecArgs &s);

}  // namespace gpe
