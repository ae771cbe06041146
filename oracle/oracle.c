/*
 * FP64 CPU oracle for the time-splitting spectral (TSSP) Gross-Pitaevskii step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this file.  It
 * shares no code, header, table or helper with the CUDA library and never
 * calls it.
 *
 * It is deliberately plain and slow: every quantity is evaluated from its
 * definition in double precision, with an own iterative radix-2 FFT, in the
 * order the method states, with no fusion, merging or reordering of steps.
 *
 * Method (quTARANG paper, "Numerical Scheme and functionalities"):
 *   non-dimensional GPE (Eq. ndGPE):  i dpsi/dt = -1/2 lap psi + V psi + g |psi|^2 psi
 *   real time   : TSSP (Bao, Jin & Markowich 2003), Strang splitting
 *                 psi <- psi exp(-i (V + g|psi|^2) dt/2)
 *                 psi_hat = FFT(psi); psi_hat <- psi_hat exp(-i |k|^2 dt/2)
 *                 psi = IFFT(psi_hat)/N
 *                 psi <- psi exp(-i (V + g|psi|^2) dt/2)     (|psi| taken afresh)
 *   imaginary time: t -> -i t in the same splitting, then the wave function is
 *                 renormalised after every step (ground-state paragraph).
 *   r_rms = (int r^2 |psi|^2 dV)^(1/2)   (Results, item 1).
 *   kinetic-energy spectra: compressible / incompressible split of the
 *                 density-weighted velocity (feature list, item 3).
 *
 * Readings where the paper is silent (each stated where it is used):
 *   - the second nonlinear half-step of a real-time step uses |psi| after the
 *     inverse FFT; in imaginary time each nonlinear half-step freezes |psi| at
 *     the start of the substep;
 *   - renormalisation target N0 (default 1) after every full step;
 *   - E = int(1/2|grad psi|^2 + V|psi|^2 + g/2|psi|^4),
 *     mu = int(1/2|grad psi|^2 + V|psi|^2 + g|psi|^4) / norm;
 *   - sigma_a = (int x_a^2 |psi|^2 / norm)^(1/2), uncentred;
 *   - spectra of u = Im(conj(psi) grad psi)/|psi|, shell n = round(|k|/dk).
 *
 * Grid: C order with x fastest, idx = x + nx*(y + ny*z); x_j = lo + j*len/n;
 * k_m = 2*pi*m/len with m in FFT order (0..n/2-1, -n/2..-1).
 * Forward transform exp(-i k x), unnormalised.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int ndim;          /* 1, 2 or 3 */
    long n[3];         /* points per axis (unused axes: 1) */
    double lo[3];      /* lower box corner */
    double len[3];     /* periodic box length */
    double g;          /* interaction parameter */
    double dt;         /* time step */
    double gamma[3];   /* V = 1/2 sum_a gamma_a^2 x_a^2 ... */
    const double *V;   /* ... unless V != NULL: V sampled at every grid point
                          (same order as psi); the model equation allows any V(r) */
} orc_grid;

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */

static long total_points(const orc_grid *G)
{
    long N = 1;
    for (int a = 0; a < G->ndim; a++) N *= G->n[a];
    return N;
}

static double cell_volume(const orc_grid *G)
{
    double dv = 1.0;
    for (int a = 0; a < G->ndim; a++) dv *= G->len[a] / (double)G->n[a];
    return dv;
}

/* coordinate of grid index j on axis a */
static double coord(const orc_grid *G, int a, long j)
{
    return G->lo[a] + (double)j * G->len[a] / (double)G->n[a];
}

/* signed FFT-order mode number of index m on an axis of n points */
static long mode_of(long m, long n) { return (m < n / 2) ? m : m - n; }

static double wavenumber(const orc_grid *G, int a, long m)
{
    return 2.0 * ORC_PI * (double)mode_of(m, G->n[a]) / G->len[a];
}

/* split a flat index into per-axis indices */
static void unflatten(const orc_grid *G, long idx, long j[3])
{
    j[0] = j[1] = j[2] = 0;
    for (int a = 0; a < G->ndim; a++) { j[a] = idx % G->n[a]; idx /= G->n[a]; }
}

/* harmonic trap V = 1/2 sum gamma_a^2 x_a^2 (paper, validation potentials) */
static double potential(const orc_grid *G, const long j[3])
{
    if (G->V) return G->V[j[0] + G->n[0] * (j[1] + G->n[1] * j[2])];
    double v = 0.0;
    for (int a = 0; a < G->ndim; a++) {
        double x = coord(G, a, j[a]);
        v += 0.5 * G->gamma[a] * G->gamma[a] * x * x;
    }
    return v;
}

static double ksq(const orc_grid *G, const long j[3])
{
    double s = 0.0;
    for (int a = 0; a < G->ndim; a++) {
        double k = wavenumber(G, a, j[a]);
        s += k * k;
    }
    return s;
}

static int is_pow2(long n) { return n >= 1 && (n & (n - 1)) == 0; }

static int check_grid(const orc_grid *G)
{
    if (G->ndim < 1 || G->ndim > 3) return -1;
    for (int a = 0; a < G->ndim; a++) {
        if (!is_pow2(G->n[a])) return -2;
        if (!(G->len[a] > 0.0)) return -3;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* radix-2 FFT                                                         */
/* ------------------------------------------------------------------ */

/* In-place iterative radix-2 Cooley-Tukey transform of one line of n = 2^p
 * points: bit-reversal permutation, then butterflies of growing span.
 * sign = -1: forward exp(-i...), sign = +1: inverse exp(+i...), both
 * unnormalised.  tw[t] = exp(sign*2*pi*i*t/n), t < n/2. */
static void fft_line(cplx *a, long n, const cplx *tw)
{
    if (n < 2) return;
    for (long i = 1, j = 0; i < n; i++) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (long span = 2; span <= n; span <<= 1) {
        long half = span / 2, step = n / span;
        for (long i = 0; i < n; i += span) {
            for (long k = 0; k < half; k++) {
                cplx u = a[i + k];
                cplx v = a[i + k + half] * tw[k * step];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
        }
    }
}

/* Multi-dimensional transform as 1D transforms along each axis in turn. */
int orc_fft(cplx *x, int ndim, const long *n, int sign)
{
    long N = 1, nn[3] = {1, 1, 1};
    for (int a = 0; a < ndim; a++) {
        if (!is_pow2(n[a])) return -2;
        nn[a] = n[a];
        N *= n[a];
    }
    long stride = 1;
    for (int a = 0; a < ndim; a++) {
        long na = nn[a];
        long lines = N / na;
        cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)(na / 2 + 1));
        for (long t = 0; t < na / 2 + 1; t++)
            tw[t] = cos(2.0 * ORC_PI * (double)t / (double)na)
                  + I * (double)sign * sin(2.0 * ORC_PI * (double)t / (double)na);
        #pragma omp parallel
        {
            cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)na);
            #pragma omp for schedule(static)
            for (long li = 0; li < lines; li++) {
                long inner = li % stride, outer = li / stride;
                long base = inner + outer * stride * na;
                for (long j = 0; j < na; j++) buf[j] = x[base + j * stride];
                fft_line(buf, na, tw);
                for (long j = 0; j < na; j++) x[base + j * stride] = buf[j];
            }
            free(buf);
        }
        free(tw);
        stride *= na;
    }
    return 0;
}

/* Brute-force O(N^2) multi-dimensional DFT, straight from the definition
 * y_k = sum_x x_j exp(sign * 2 pi i sum_a k_a j_a / n_a).  Tiny grids only. */
int orc_dft_brute(const cplx *x, cplx *y, int ndim, const long *n, int sign)
{
    long nn[3] = {1, 1, 1}, N = 1;
    for (int a = 0; a < ndim; a++) { nn[a] = n[a]; N *= n[a]; }
    for (long kk = 0; kk < N; kk++) {
        long k0 = kk % nn[0], k1 = (kk / nn[0]) % nn[1], k2 = kk / (nn[0] * nn[1]);
        cplx s = 0.0;
        for (long jj = 0; jj < N; jj++) {
            long j0 = jj % nn[0], j1 = (jj / nn[0]) % nn[1], j2 = jj / (nn[0] * nn[1]);
            /* phase in turns, reduced exactly with integers before scaling */
            double ph = (double)((k0 * j0) % nn[0]) / (double)nn[0]
                      + (double)((k1 * j1) % nn[1]) / (double)nn[1]
                      + (double)((k2 * j2) % nn[2]) / (double)nn[2];
            s += x[jj] * (cos(2.0 * ORC_PI * ph) + I * (double)sign * sin(2.0 * ORC_PI * ph));
        }
        y[kk] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* TSSP substeps                                                       */
/* ------------------------------------------------------------------ */

/* Real-time nonlinear substep: psi <- psi exp(-i (V + g|psi|^2) tau).
 * |psi| is unchanged by it, so the substep is the exact solution of
 * i dpsi/dt = (V + g|psi|^2) psi over tau (Eq. ndGPE without the Laplacian). */
static void nonlinear_real(cplx *psi, const orc_grid *G, double tau)
{
    long N = total_points(G);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double rho = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        double th = (potential(G, j) + G->g * rho) * tau;
        psi[i] *= cos(th) - I * sin(th);
    }
}

/* Real-time kinetic substep in Fourier space: psi_hat <- psi_hat exp(-i |k|^2 tau / 2). */
static void kinetic_real(cplx *ph, const orc_grid *G, double tau)
{
    long N = total_points(G);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double th = 0.5 * ksq(G, j) * tau;
        ph[i] *= cos(th) - I * sin(th);
    }
}

/* Imaginary-time nonlinear substep (t -> -i t): psi <- psi exp(-(V + g|psi|^2) tau),
 * with |psi| frozen at the start of the substep. */
static void nonlinear_imag(cplx *psi, const orc_grid *G, double tau)
{
    long N = total_points(G);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double rho = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        psi[i] *= exp(-(potential(G, j) + G->g * rho) * tau);
    }
}

/* Imaginary-time kinetic substep: psi_hat <- psi_hat exp(-|k|^2 tau / 2). */
static void kinetic_imag(cplx *ph, const orc_grid *G, double tau)
{
    long N = total_points(G);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        ph[i] *= exp(-0.5 * ksq(G, j) * tau);
    }
}

static void scale_all(cplx *x, long N, double s)
{
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) x[i] *= s;
}

static double norm_of(const cplx *psi, const orc_grid *G)
{
    long N = total_points(G);
    double s = 0.0;
    for (long i = 0; i < N; i++)
        s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s * cell_volume(G);
}

/* One real-time TSSP step (Strang splitting, halves not merged). */
static void step_real_once(cplx *psi, const orc_grid *G)
{
    long N = total_points(G);
    nonlinear_real(psi, G, 0.5 * G->dt);
    orc_fft(psi, G->ndim, G->n, -1);
    kinetic_real(psi, G, G->dt);
    orc_fft(psi, G->ndim, G->n, +1);
    scale_all(psi, N, 1.0 / (double)N);
    nonlinear_real(psi, G, 0.5 * G->dt);
}

int orc_step_real(cplx *psi, const orc_grid *G, long nsteps)
{
    int e = check_grid(G);
    if (e) return e;
    for (long s = 0; s < nsteps; s++) step_real_once(psi, G);
    return 0;
}

/* Real-time steps in a harmonic trap whose frequencies change in time
 * (Eq. ndGPE with V(r, t); the paper lists time-dependent potentials among
 * the solver's functionalities).  gamma_t holds (nsteps + 1) rows of three
 * trap frequencies, the trap at the time levels t_0 .. t_nsteps of the call.
 * Step n runs the Strang splitting of step_real_once with the first nonlinear
 * half-step in the trap of t_n and the second in the trap of t_{n+1}, so each
 * nonlinear half-step evaluates V at the end of the time interval it is
 * adjacent to, and the scheme stays symmetric in time.  The sampled
 * potential G->V, if any, is not used (the schedule is the potential). */
int orc_step_real_trap(cplx *psi, const orc_grid *G, long nsteps, const double *gamma_t)
{
    int e = check_grid(G);
    if (e) return e;
    if (!gamma_t) return -1;
    orc_grid H = *G;
    H.V = NULL;
    long N = total_points(G);
    for (long s = 0; s < nsteps; s++) {
        for (int a = 0; a < 3; a++) H.gamma[a] = a < G->ndim ? gamma_t[3 * s + a] : 0.0;
        nonlinear_real(psi, &H, 0.5 * G->dt);
        orc_fft(psi, G->ndim, G->n, -1);
        kinetic_real(psi, &H, G->dt);
        orc_fft(psi, G->ndim, G->n, +1);
        scale_all(psi, N, 1.0 / (double)N);
        for (int a = 0; a < 3; a++) H.gamma[a] = a < G->ndim ? gamma_t[3 * (s + 1) + a] : 0.0;
        nonlinear_real(psi, &H, 0.5 * G->dt);
    }
    return 0;
}

/* One imaginary-time step followed by renormalisation to N0. */
static int step_imag_once(cplx *psi, const orc_grid *G, double N0)
{
    long N = total_points(G);
    nonlinear_imag(psi, G, 0.5 * G->dt);
    orc_fft(psi, G->ndim, G->n, -1);
    kinetic_imag(psi, G, G->dt);
    orc_fft(psi, G->ndim, G->n, +1);
    scale_all(psi, N, 1.0 / (double)N);
    nonlinear_imag(psi, G, 0.5 * G->dt);
    double nrm = norm_of(psi, G);
    if (!(nrm > 0.0) || !isfinite(nrm)) return -5;
    scale_all(psi, N, sqrt(N0 / nrm));
    return 0;
}

int orc_step_imag(cplx *psi, const orc_grid *G, long nsteps, double N0)
{
    int e = check_grid(G);
    if (e) return e;
    for (long s = 0; s < nsteps; s++) {
        e = step_imag_once(psi, G, N0);
        if (e) return e;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* diagnostics                                                         */
/* ------------------------------------------------------------------ */

/* out = {norm, E_kin, E_pot, E_int, E, mu}.  Gradients are spectral:
 * int |grad psi|^2 dV = dV/N sum_k |k|^2 |psi_hat_k|^2 (Parseval). */
int orc_norm_energy(const cplx *psi, const orc_grid *G, double *out)
{
    int e = check_grid(G);
    if (e) return e;
    long N = total_points(G);
    double dv = cell_volume(G);
    double nrm = 0.0, epot = 0.0, eint = 0.0, ekin = 0.0;
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double rho = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        nrm += rho;
        epot += potential(G, j) * rho;
        eint += 0.5 * G->g * rho * rho;
    }
    cplx *ph = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    if (!ph) return -4;
    memcpy(ph, psi, sizeof(cplx) * (size_t)N);
    orc_fft(ph, G->ndim, G->n, -1);
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double a2 = creal(ph[i]) * creal(ph[i]) + cimag(ph[i]) * cimag(ph[i]);
        ekin += 0.5 * ksq(G, j) * a2;
    }
    free(ph);
    nrm *= dv;
    epot *= dv;
    eint *= dv;
    ekin *= dv / (double)N;
    out[0] = nrm;
    out[1] = ekin;
    out[2] = epot;
    out[3] = eint;
    out[4] = ekin + epot + eint;
    out[5] = (ekin + epot + 2.0 * eint) / nrm;
    return 0;
}

/* out = {sigma_x, sigma_y, sigma_z, r_rms}; sigma_a^2 = int x_a^2|psi|^2 / norm,
 * r_rms^2 = sum_a sigma_a^2 (unused axes report 0). */
int orc_rms(const cplx *psi, const orc_grid *G, double *out)
{
    int e = check_grid(G);
    if (e) return e;
    long N = total_points(G);
    double m2[3] = {0, 0, 0}, nrm = 0.0;
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double rho = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        nrm += rho;
        for (int a = 0; a < G->ndim; a++) {
            double x = coord(G, a, j[a]);
            m2[a] += x * x * rho;
        }
    }
    double r2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double s2 = (a < G->ndim) ? m2[a] / nrm : 0.0;
        out[a] = sqrt(s2);
        r2 += s2;
    }
    out[3] = sqrt(r2);
    return 0;
}

/* Imaginary-time run to the ground state: steps in chunks of check_every,
 * stopping once |E(now) - E(previous check)| < etol (absolute), the first
 * reference being the energy of the input state. */
int orc_ground(cplx *psi, const orc_grid *G, long max_steps, double N0, double etol,
               long check_every, long *steps_done, double *E_final)
{
    int e = check_grid(G);
    if (e) return e;
    if (check_every < 1) return -1;
    double o[6];
    orc_norm_energy(psi, G, o);
    double eprev = o[4];
    long done = 0;
    while (done < max_steps) {
        long chunk = check_every;
        if (chunk > max_steps - done) chunk = max_steps - done;
        e = orc_step_imag(psi, G, chunk, N0);
        if (e) return e;
        done += chunk;
        orc_norm_energy(psi, G, o);
        if (fabs(o[4] - eprev) < etol) { eprev = o[4]; break; }
        eprev = o[4];
    }
    *steps_done = done;
    *E_final = eprev;
    return 0;
}

/* Shell index of a wave vector: n = round(|k| / dk), dk = 2 pi / max_a len_a,
 * evaluated as sqrt(sum_a (m_a * Lmax / len_a)^2) so that cubic boxes use
 * integer mode numbers only. */
static long shell_of(const orc_grid *G, const long j[3])
{
    double lmax = 0.0;
    for (int a = 0; a < G->ndim; a++) if (G->len[a] > lmax) lmax = G->len[a];
    double q2 = 0.0;
    for (int a = 0; a < G->ndim; a++) {
        double q = (double)mode_of(j[a], G->n[a]) * (lmax / G->len[a]);
        q2 += q * q;
    }
    return (long)floor(sqrt(q2) + 0.5);
}

long orc_spectrum_nshells(const orc_grid *G)
{
    if (check_grid(G)) return -1;
    long j[3] = {0, 0, 0};
    for (int a = 0; a < G->ndim; a++) j[a] = G->n[a] / 2;   /* mode -n/2: largest |m| */
    return shell_of(G, j) + 1;
}

/* Kinetic-energy spectra (feature list, item 3):
 *   d_a psi = IFFT(i k_a psi_hat)/N with the Nyquist mode of i k_a set to 0;
 *   u_a = Im(conj(psi) d_a psi)/|psi| (0 where |psi|^2 < 1e-30);
 *   u_hat = FFT(u); u_c = k (k.u_hat)/|k|^2 (0 at k = 0); u_i = u_hat - u_c;
 *   E_i(n) = 1/2 sum_{shell n} |u_i|^2 dV/N, E_c(n) likewise.
 * e_inc / e_comp may be NULL; each has nshells entries. */
int orc_spectrum(const cplx *psi, const orc_grid *G, double *e_inc, double *e_comp, long nshells)
{
    int e = check_grid(G);
    if (e) return e;
    long need = orc_spectrum_nshells(G);
    if (nshells < need) return -1;
    long N = total_points(G);
    int d = G->ndim;
    double dv = cell_volume(G);
    cplx *ph = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *uh[3] = {NULL, NULL, NULL};
    if (!ph) return -4;
    memcpy(ph, psi, sizeof(cplx) * (size_t)N);
    orc_fft(ph, d, G->n, -1);
    for (int a = 0; a < d; a++) {
        uh[a] = (cplx *)malloc(sizeof(cplx) * (size_t)N);
        if (!uh[a]) return -4;
        /* derivative along a */
        for (long i = 0; i < N; i++) {
            long j[3];
            unflatten(G, i, j);
            double k = (2 * j[a] == G->n[a]) ? 0.0 : wavenumber(G, a, j[a]);
            uh[a][i] = I * k * ph[i];
        }
        orc_fft(uh[a], d, G->n, +1);
        for (long i = 0; i < N; i++) {
            cplx dpsi = uh[a][i] / (double)N;
            double rho = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
            double u = 0.0;
            if (rho >= 1e-30) u = cimag(conj(psi[i]) * dpsi) / sqrt(rho);
            uh[a][i] = u;
        }
        orc_fft(uh[a], d, G->n, -1);
    }
    if (e_inc) memset(e_inc, 0, sizeof(double) * (size_t)nshells);
    if (e_comp) memset(e_comp, 0, sizeof(double) * (size_t)nshells);
    for (long i = 0; i < N; i++) {
        long j[3];
        unflatten(G, i, j);
        double kv[3] = {0, 0, 0}, k2 = 0.0;
        for (int a = 0; a < d; a++) { kv[a] = wavenumber(G, a, j[a]); k2 += kv[a] * kv[a]; }
        cplx kdotu = 0.0;
        for (int a = 0; a < d; a++) kdotu += kv[a] * uh[a][i];
        double ec = 0.0, ei = 0.0;
        for (int a = 0; a < d; a++) {
            cplx uc = (k2 > 0.0) ? kv[a] * kdotu / k2 : 0.0;
            cplx ui = uh[a][i] - uc;
            ec += creal(uc) * creal(uc) + cimag(uc) * cimag(uc);
            ei += creal(ui) * creal(ui) + cimag(ui) * cimag(ui);
        }
        long sh = shell_of(G, j);
        if (e_inc) e_inc[sh] += 0.5 * ei * dv / (double)N;
        if (e_comp) e_comp[sh] += 0.5 * ec * dv / (double)N;
    }
    for (int a = 0; a < d; a++) free(uh[a]);
    free(ph);
    return 0;
}

/* Quantum-pressure and particle-number spectra (the decomposition of the
 * kinetic energy in the feature list, item 3, completed by its third part):
 *   w_a = Re(conj(psi) d_a psi)/|psi| = d_a |psi| (0 where |psi|^2 < 1e-30),
 *   E_qp(n) = 1/2 sum_{shell n} sum_a |FFT(w_a)|^2 dV/N;
 *   N(n) = sum_{shell n} |psi_hat|^2 dV/N   (sum over shells = norm).
 * d_a psi as in orc_spectrum.  e_qp / n_num may be NULL. */
int orc_spectrum_qp_num(const cplx *psi, const orc_grid *G, double *e_qp, double *n_num, long nshells)
{
    int e = check_grid(G);
    if (e) return e;
    long need = orc_spectrum_nshells(G);
    if (nshells < need) return -1;
    long N = total_points(G);
    int d = G->ndim;
    double dv = cell_volume(G);
    cplx *ph = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *wh = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    if (!ph || !wh) return -4;
    memcpy(ph, psi, sizeof(cplx) * (size_t)N);
    orc_fft(ph, d, G->n, -1);
    if (e_qp) memset(e_qp, 0, sizeof(double) * (size_t)nshells);
    if (n_num) memset(n_num, 0, sizeof(double) * (size_t)nshells);
    if (n_num) {
        for (long i = 0; i < N; i++) {
            long j[3];
            unflatten(G, i, j);
            n_num[shell_of(G, j)] += (creal(ph[i]) * creal(ph[i]) + cimag(ph[i]) * cimag(ph[i])) * dv / (double)N;
        }
    }
    if (e_qp) {
        for (int a = 0; a < d; a++) {
            for (long i = 0; i < N; i++) {
                long j[3];
                unflatten(G, i, j);
                double k = (2 * j[a] == G->n[a]) ? 0.0 : wavenumber(G, a, j[a]);
                wh[i] = I * k * ph[i];
            }
            orc_fft(wh, d, G->n, +1);
            for (long i = 0; i < N; i++) {
                cplx dpsi = wh[i] / (double)N;
                double rho = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
                double w = 0.0;
                if (rho >= 1e-30) w = creal(conj(psi[i]) * dpsi) / sqrt(rho);
                wh[i] = w;
            }
            orc_fft(wh, d, G->n, -1);
            for (long i = 0; i < N; i++) {
                long j[3];
                unflatten(G, i, j);
                e_qp[shell_of(G, j)] += 0.5 * (creal(wh[i]) * creal(wh[i]) + cimag(wh[i]) * cimag(wh[i])) * dv / (double)N;
            }
        }
    }
    free(wh);
    free(ph);
    return 0;
}

/* thread control for the timed CPU baseline */
int orc_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}
