/*
 * gpe.h - C ABI of the GB300 time-splitting spectral (TSSP) Gross-Pitaevskii library.
 *
 * The library advances solutions of the non-dimensional Gross-Pitaevskii
 * equation (quTARANG paper, Eq. ndGPE)
 *
 *     i dpsi/dt = -1/2 lap psi + V psi + g |psi|^2 psi,
 *
 * with V = 1/2 sum_a gamma_a^2 x_a^2 or any V sampled on the grid (V_host),
 * on periodic grids in 1, 2 or 3 dimensions with the TSSP scheme the paper
 * uses ("Numerical Scheme and functionalities": TSSP for dynamics, the same
 * scheme in imaginary time t -> -i t with renormalisation after every step for
 * ground states), and evaluates the norm, energy, chemical potential, rms sizes
 * (Results, item 1) and the compressible / incompressible kinetic-energy
 * spectra (feature list, item 3), completed by the quantum-pressure and
 * particle-number spectra.
 *
 * Conventions shared by every entry point
 *   Grid      n[a] points on axis a (powers of two, 2..4096; unused axes 1),
 *             periodic box [lo[a], lo[a] + len[a]), x_j = lo + j*len/n.
 *   Layout    psi is interleaved complex (re, im), C order with x fastest:
 *             element (x, y, z) of instance b sits at b*N + x + n0*(y + n1*z),
 *             N = n0*n1*n2.  complex64 (GPE_C64, 8 bytes per point) or
 *             complex128 (GPE_C128, 16 bytes).  Device pointers are CUDA
 *             device memory owned by the caller, 16-byte aligned.
 *   Streams   every call is enqueued on the stream given to gpe_plan_create
 *             (NULL: the legacy default stream).  Calls that return values to
 *             host memory synchronise that stream before returning.
 *   Errors    every call returns a gpe_status and never aborts the process;
 *             gpe_last_error() gives a message for the calling thread.
 *   Ownership a plan owns its tables, workspace and partial-sum buffers; the
 *             caller owns psi.  Plans are not thread safe: use one per thread.
 */
#ifndef GPE_H
#define GPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gpe_status {
    GPE_OK = 0,
    GPE_EINVAL = 1,        /* bad argument (NULL pointer, bad size, bad flag)   */
    GPE_EUNSUPPORTED = 2,  /* grid not supported (non power of two, >4096, ndim) */
    GPE_ENOMEM = 3,        /* device or host allocation failed                  */
    GPE_ECUDA = 4,         /* a CUDA runtime call failed                        */
    GPE_ENUMERIC = 5,      /* non-finite or zero norm met                       */
    GPE_ETIMEOUT = 6,      /* a wait ran past its limit                         */
    GPE_EBUSY = 7,         /* admission refused: budget or slots exhausted      */
    GPE_ENOTREADY = 8      /* polled request not finished yet                   */
} gpe_status;

typedef enum gpe_precision {
    GPE_C64 = 0,   /* complex64 bulk arithmetic, FP64 reductions and tables */
    GPE_C128 = 1   /* complex128 throughout                                 */
} gpe_precision;

/* Problem description (copied by gpe_plan_create). */
typedef struct gpe_plan_desc {
    int ndim;                   /* 1, 2 or 3                                        */
    int64_t n[3];               /* points per axis, x first; unused axes ignored    */
    double lo[3];               /* box corner                                        */
    double len[3];              /* box length (> 0)                                  */
    double g;                   /* interaction parameter                             */
    double dt;                  /* time step (negative allowed: backward in time)    */
    double gamma[3];            /* trap frequencies, V = 1/2 sum gamma_a^2 x_a^2      */
    int prec;                   /* gpe_precision                                     */
    int batch;                  /* instances stored back to back (>= 1)              */
    const double *g_each;       /* host, batch entries overriding g, or NULL         */
    const double *gamma_each;   /* host, batch*3 entries overriding gamma, or NULL   */
    const double *V_host;       /* host, N values of a potential sampled at the grid
                                   points (layout of one instance), shared by all
                                   instances and used instead of the harmonic trap
                                   (gamma and gamma_each must then be zero / NULL);
                                   or NULL.  The model equation allows any V(r);
                                   copied at plan creation.                         */
} gpe_plan_desc;

typedef struct gpe_plan gpe_plan;

/* Validate desc, build the per-axis twiddle, kinetic-phase and trap-phase
 * tables (evaluated in FP64 on the host) and allocate workspace.
 * cuda_stream: a cudaStream_t or NULL.  On success *out owns everything. */
gpe_status gpe_plan_create(const gpe_plan_desc *desc, void *cuda_stream, gpe_plan **out);
gpe_status gpe_plan_destroy(gpe_plan *plan);

/* Advance every instance by nsteps real-time TSSP steps in place (Numerical
 * Scheme: TSSP of Bao et al.): per step
 *   psi <- psi exp(-i (V + g|psi|^2) dt/2); psi_hat = FFT psi;
 *   psi_hat <- psi_hat exp(-i |k|^2 dt/2); psi = IFFT(psi_hat)/N;
 *   psi <- psi exp(-i (V + g|psi|^2) dt/2).
 * Consecutive nonlinear half-steps are merged into one full step (exact:
 * |psi| does not change under them).  psi_dev is real-space on entry and
 * on return.  nsteps >= 0. */
gpe_status gpe_step_real(gpe_plan *plan, void *psi_dev, int64_t nsteps);

/* gpe_step_real in a harmonic trap whose frequencies change in time, V(r, t) =
 * sum_a gamma_a(t)^2 x_a^2 / 2 (Eq. ndGPE allows any V; the paper lists
 * time-dependent potentials among the solver's functionalities).  gamma_host
 * holds (nsteps + 1) rows of three frequencies (x, y, z; axes beyond ndim are
 * ignored): row n is the trap at time level n of this call, t_n = n dt.  Step
 * n applies its first nonlinear half-step in the trap of row n and its second
 * in the trap of row n + 1 (merged with the next step's first half, exact as in
 * gpe_step_real); the kinetic substep is unchanged.  The schedule replaces the
 * plan's own trap for this call, on every axis and every instance, and any
 * axis may be trapped.  A step change of gamma between two rows is a quench at
 * that time level.  The tables of each time level are built on the device
 * (host memory is read only during the call).  Diagnostics afterwards still use
 * the plan's own trap.  GPE_EUNSUPPORTED for plans with V_host; GPE_EINVAL for
 * NULL or non-finite frequencies or nsteps < 0. */
gpe_status gpe_step_real_trap(gpe_plan *plan, void *psi_dev, int64_t nsteps, const double *gamma_host);

/* Same as gpe_step_real on a HOST buffer: copies psi in (pageable or pinned),
 * steps on the device and copies the result back.  Uses plan workspace.  For
 * one instance of at least 64 MiB in pinned host memory (2D/3D, no sampled
 * potential) the copies go in slabs of planes of the slowest axis on a second
 * stream and overlap the sweeps that stay inside a slab; results are the same
 * bits either way.  Returns when psi_host holds the result. */
gpe_status gpe_step_real_host(gpe_plan *plan, void *psi_host, int64_t nsteps);

/* Imaginary-time TSSP (ground-state paragraph: t -> -i t, renormalise each
 * step): per step psi <- psi exp(-(V + g|psi|^2) dt/2) (|psi| frozen at the
 * substep start), FFT, exp(-|k|^2 dt/2), IFFT/N, the same half-step again,
 * then psi <- psi sqrt(target_norm / norm).  Runs in chunks of check_every
 * steps and stops after a chunk once |E - E_previous_check| < etol for every
 * instance (etol <= 0: never stops early), or after max_steps.  The first
 * reference energy is that of the input.  steps_done (may be NULL) receives
 * the steps taken; E_final (may be NULL) receives batch energies.  The test
 * runs on the device after each chunk; the host enqueues chunks a window at a
 * time (2, 4, 8, then 16 chunks) and reads the stop word once per window, and
 * the kernels of chunks queued after the test fired do nothing, so results
 * are those of the check that stopped the run.  A zero or non-finite norm or
 * energy returns GPE_ENUMERIC (detected at the end of its window). */
gpe_status gpe_step_imag(gpe_plan *plan, void *psi_dev, int64_t max_steps, double target_norm,
                         double etol, int check_every, int64_t *steps_done, double *E_final);

/* out_host[6*b + i], i = norm, E_kin, E_pot, E_int, E, mu for instance b:
 *   norm = sum|psi|^2 dV, E_kin = 1/2 sum_k |k|^2 |psi_hat|^2 dV/N,
 *   E_pot = sum V|psi|^2 dV, E_int = g/2 sum|psi|^4 dV, E = sum of the three,
 *   mu = (E_kin + E_pot + 2 E_int)/norm.  Reductions in FP64. */
gpe_status gpe_norm_energy(gpe_plan *plan, const void *psi_dev, double *out_host);

/* out_host[4*b + i] = sigma_x, sigma_y, sigma_z, r_rms for instance b:
 * sigma_a^2 = sum x_a^2|psi|^2 / sum|psi|^2 (uncentred), r_rms^2 = sum sigma_a^2
 * (Results, item 1: r_rms = (int r^2 |psi|^2 dV)^(1/2) for unit norm). */
gpe_status gpe_rms_size(gpe_plan *plan, const void *psi_dev, double *out_host);

/* Kinetic-energy spectra (feature list, item 3).  u_a = Im(conj(psi) d_a psi)/|psi|
 * with spectral derivatives (Nyquist mode of i k_a zeroed, u = 0 where
 * |psi|^2 < 1e-30); u_hat = FFT u split into u_c = k(k.u_hat)/|k|^2 and
 * u_i = u_hat - u_c; E(n) = 1/2 sum over shell n of |u|^2 dV/N with
 * n = round(|k| / dk), dk = 2 pi / max_a len_a.
 * The kinetic energy splits further into a quantum-pressure part:
 * GPE_SPEC_QP bins 1/2 sum_a |FFT w_a|^2 dV/N with w_a = Re(conj(psi) d_a psi)/|psi|
 * = d_a |psi|, so that INC + COMP + QP summed over shells is E_kin for fields
 * without Nyquist content; GPE_SPEC_NUM bins the particle number
 * |psi_hat|^2 dV/N (its sum is the norm).
 * kinds: any non-empty combination of GPE_SPEC_INC, GPE_SPEC_COMP,
 * GPE_SPEC_QP, GPE_SPEC_NUM.  out_host receives, for each requested kind in
 * that order, nshells doubles per instance ([kind][b][shell]).
 * nshells must be >= gpe_spectrum_nshells(plan). */
#define GPE_SPEC_INC 1u
#define GPE_SPEC_COMP 2u
#define GPE_SPEC_QP 4u
#define GPE_SPEC_NUM 8u
int64_t gpe_spectrum_nshells(const gpe_plan *plan);
gpe_status gpe_spectrum(gpe_plan *plan, const void *psi_dev, unsigned kinds, double *out_host,
                        int64_t nshells);

/* Plan options (implementation choices, no counterpart in the paper).  Every
 * option takes 0 or 1; results are bit-identical for every setting (each
 * line's arithmetic does not depend on them, with the one exception noted at
 * GPE_OPT_GENERIC_PASSES), only the speed changes.
 *   GPE_OPT_TMA_STAGING  1 (default): tiles of the y and z sweeps are fetched
 *                        by the tensor-memory accelerator when the grid allows
 *                        it (n0 a multiple of the tile's line count, instances
 *                        back to back in one array); 0: by per-thread
 *                        asynchronous copies.  Sets both axes; GPE_OPT_TMA_Y /
 *                        GPE_OPT_TMA_Z set one.
 *   GPE_OPT_TILE_X/Y/Z   tile shape of the sweeps along x, y, z (0 default,
 *                        1 the alternative compiled shape: different lines per
 *                        tile and CTAs per SM).
 *   GPE_OPT_GENERIC_PASSES  1: every sweep runs the generic pass kernel, which
 *                        reads its program (pointwise ops, transforms,
 *                        reduction) from the launch arguments; 0 (default):
 *                        the sweeps of the real- and imaginary-time steps on
 *                        complex64 lines of 256 to 1024 points run kernels
 *                        compiled for their program.  For tests and timing.
 *                        The one exception to bit-identical results: with
 *                        this option imaginary-time steps can differ in the
 *                        last place (real-time steps do not).
 *   GPE_OPT_NO_DITHER    1: turns off the phase dither of complex64
 *                        real-time steps (the default, 0, keeps it): each
 *                        step's kinetic substep also turns the state by a
 *                        global phase of at most 0.01 rad and the nonlinear
 *                        substep of the same step turns it back, which changes
 *                        the results by rounding only and keeps the rounding
 *                        errors of slowly turning modes from adding up
 *                        coherently (norm drift).  Unlike the options above
 *                        it changes the bits of complex64 results.
 *   GPE_OPT_LINE_CLUSTER 1 (default): complex128 real-time steps of 1D
 *                        plans with lines of 64, 128 or 256 points and at
 *                        most 32 instances spread each line over a cluster
 *                        of 4, 8 or 16 CTAs (a latency path: FP64 work on
 *                        one SM is slow on this GPU); 0: one CTA per line.
 *                        The two factor the transform differently, so their
 *                        results differ in rounding (both agree with the
 *                        FP64 reference to about 1e-14 per step).
 *   GPE_OPT_TEST_STALL_COPIES  test hook for the failure handling: 1 makes
 *                        every copy-engine tile wait, and every exchange wait
 *                        of the 1D cluster kernel, expect 16 bytes more than
 *                        arrive, so the wait runs out after its limit (about
 *                        2 s), the kernel abandons its work, and the next
 *                        synchronising call returns GPE_ETIMEOUT.  Results of
 *                        such a launch are undefined.
 * gpe_plan_set_option returns GPE_EINVAL for an unknown option or value and
 * takes effect at the next launch; gpe_plan_get_option reads one back. */
enum gpe_option {
    GPE_OPT_TMA_STAGING = 1,
    GPE_OPT_TILE_X = 2,
    GPE_OPT_TILE_Y = 3,
    GPE_OPT_TILE_Z = 4,
    GPE_OPT_TMA_Y = 5,
    GPE_OPT_TMA_Z = 6,
    GPE_OPT_GENERIC_PASSES = 7,
    GPE_OPT_NO_DITHER = 8,
    GPE_OPT_LINE_CLUSTER = 9,
    GPE_OPT_TEST_STALL_COPIES = 99
};
gpe_status gpe_plan_set_option(gpe_plan *plan, int option, int64_t value);
gpe_status gpe_plan_get_option(const gpe_plan *plan, int option, int64_t *value);

/* Autotuner (no counterpart in the paper): for every axis the plan sweeps, in
 * the step's order and twice over, times each tile shape (and, on y/z, each staging mode
 * unless GPE_TUNE_NO_TMA) as whole steady real-time steps with the other axes
 * at their current choice (from psi_dev, or zeros when psi_dev is NULL,
 * advanced through a call's prologue; the caller's array is only read),
 * `reps` samples per candidate taken round-robin across the candidates (a
 * sample is one step, or several on grids whose step is shorter than about
 * 2 ms), and keeps the candidate with the fastest sample.  Choices are remembered per
 * grid, precision and instance count for the life of the process, so later
 * plans of the same shape tune without timing.  Needs two state-sized device
 * scratch arrays for the duration of the call; synchronises the plan stream.
 * 1D plans have nothing to tune (GPE_OK). */
#define GPE_TUNE_NO_TMA 1
gpe_status gpe_plan_autotune(gpe_plan *plan, const void *psi_dev, int reps, int flags);

/* Tracing (profiling aid, no counterpart in the paper).  While enabled, every
 * kernel launch the plan makes is bracketed by two CUDA events on the plan
 * stream and filed under a kind such as "x512:I-NR-F" (axis, line length, and
 * the pass's substeps: F/I forward/inverse FFT, NR/NI nonlinear real/imaginary,
 * KR/KI kinetic real/imaginary, S scale, diag/red reductions).  Enabling clears
 * earlier records.  gpe_trace_read synchronises the stream and returns, for
 * kind i < gpe_trace_count(), its name (NUL-terminated, truncated to name_len),
 * the number of launches and their summed device time in milliseconds. */
gpe_status gpe_trace_enable(gpe_plan *plan, int enable);
int gpe_trace_count(gpe_plan *plan);
gpe_status gpe_trace_read(gpe_plan *plan, int i, char *name, size_t name_len, int64_t *launches,
                          double *total_ms);

/* Norm and energy without any allocation (the paper has no counterpart; this
 * exists for callers that cannot allocate).  Some callers cannot call
 * cudaMalloc: code that runs under a framework owning all device memory through
 * its own allocator, and latency-critical loops where cudaMalloc/cudaFree
 * would synchronise the device.  For one instance described by desc (batch
 * must be 1; g_each and gamma_each are ignored) this computes the six values
 * of gpe_norm_energy into out_host[0..5] using only psi_dev, out_host and a
 * fixed device array of about 2.4 MiB that every GPU loading the library
 * holds until the process exits; it calls no allocating routine.
 * Limit: N / n[a] <= GPE_NOALLOC_MAX_LINES on every axis (for example 1024^2,
 * 4096 x 32, 128^3); larger grids, and descriptions with V_host, are rejected
 * with GPE_EUNSUPPORTED.
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, which allocates nothing once the library's device
 * code is loaded).  With lazy module loading (the CUDA default) the first call
 * on a device loads this library's device code there, which is when the array
 * and the code take their device memory, outside any framework's allocator:
 * a framework-managed caller should make one call during its set-up.
 * The call ends with a device-to-host copy into out_host and synchronises
 * cuda_stream, so it must not be called while that stream is being captured.
 * Every call reuses the same array, so calls that overlap on the GPU (from
 * other streams or threads) race: serialise them.
 * The twiddles of its transforms are evaluated on the device, those of a plan
 * on the host, so the results can differ from gpe_norm_energy's in the last
 * place. */
#define GPE_NOALLOC_MAX_LINES 32768
gpe_status gpe_norm_energy_noalloc(const gpe_plan_desc *desc, const void *psi_dev, void *cuda_stream,
                                   double *out_host);

/* Measured double-precision FMA throughput of the current device (a
 * measurement aid for the roofline of complex128 runs, which are bound by
 * FP64 arithmetic rather than HBM; no counterpart in the paper).  Launches a
 * kernel of independent FMA chains on every SM on cuda_stream, synchronises
 * it, and writes the best of three timed launches to *flops_per_s (2 flops
 * per FMA).  GPE_EINVAL for a NULL pointer, GPE_ECUDA on a launch error. */
gpe_status gpe_measure_fp64_peak(void *cuda_stream, double *flops_per_s);

/* Thread-local message describing the last error (never NULL). */
const char *gpe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GPE_H */
