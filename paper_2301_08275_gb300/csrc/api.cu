// api.cu - plan objects and the C ABI entry points declared in include/gpe.h.
//
// A plan holds, per axis, the twiddle table exp(-2 pi i t/n), the kinetic
// substep table exp(-i k^2 dt/2) - 1 (real time) and exp(-k^2 dt/2)/n
// (imaginary time), and per instance the trap tables exp(-i V_a dt/2) - 1,
// exp(-i V_a dt) - 1 and exp(-V_a dt/2) with V_a = gamma_a^2 x^2 / 2.  All are
// evaluated in double precision on the host; in single precision the complex
// entries are stored as hi + lo float pairs (see fft_tile.cuh).  Because the
// trap is separable, V enters every nonlinear substep as a product of per-axis
// unit phases and only the g|psi|^2 part of the angle is evaluated per point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gpe.h"
#include "gpe_internal.h"

namespace gpe {
cudaError_t launch_pass_f32(bool rows, int var, const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap);
cudaError_t launch_pass_f64(bool rows, int var, const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap);
cudaError_t launch_line1d_f32(const Line1DArgs &a, cudaStream_t st);
cudaError_t launch_line1d_f64(const Line1DArgs &a, cudaStream_t st);
int lines_per_tile_f32(bool rows, int n, int var);
int lines_per_tile_f64(bool rows, int n, int var);

cudaError_t launch_pass(int prec, bool rows, const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap, int var)
{
    return prec == GPE_C64 ? launch_pass_f32(rows, var, a, st, tmap) : launch_pass_f64(rows, var, a, st, tmap);
}
int pass_lines_per_tile(int prec, bool rows, int n, int var)
{
    return prec == GPE_C64 ? lines_per_tile_f32(rows, n, var) : lines_per_tile_f64(rows, n, var);
}
cudaError_t launch_line1d(int prec, const Line1DArgs &a, cudaStream_t st)
{
    if (prec == GPE_C128 && a.cluster && line1d_cluster_applies(a)) {
        const cudaError_t e = launch_line1d_cluster(a, st);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();   // no cluster of that size fits: the one-CTA-per-line kernel
    }
    return prec == GPE_C64 ? launch_line1d_f32(a, st) : launch_line1d_f64(a, st);
}
}  // namespace gpe

using namespace gpe;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error = "no error";

static gpe_status fail(gpe_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

#define GPE_CUDA(call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? GPE_ENOMEM : GPE_ECUDA,                \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

#define GPE_TRY(expr)                         \
    do {                                      \
        gpe_status s_ = (expr);               \
        if (s_ != GPE_OK) return s_;          \
    } while (0)

extern "C" const char *gpe_last_error(void) { return g_last_error.c_str(); }

void gpe::set_last_error(const char *msg) { g_last_error = msg; }

// ------------------------------------------------------------------ plan
struct gpe_plan {
    int ndim = 0;
    int64_t n[3] = {1, 1, 1};
    int64_t N = 1;
    int64_t batch = 1;
    int prec = GPE_C64;
    size_t csize = 8, rsize = 4;
    double lo[3] = {0, 0, 0}, len[3] = {1, 1, 1}, h[3] = {0, 0, 0}, kf[3] = {0, 0, 0};
    double dt = 0, dv = 1;
    cudaStream_t st = nullptr;
    int device = 0;
    bool trap[3] = {false, false, false};
    void *tw[3] = {}, *kt[3] = {}, *ki[3] = {}, *vh[3] = {}, *vf[3] = {}, *vi[3] = {};
    void *vsamp = nullptr;       // sampled potential [N] in the bulk real type, or NULL
    double *g_dev = nullptr, *gamma_dev = nullptr, *scale = nullptr, *partials = nullptr;
    double *sums = nullptr, *out6 = nullptr, *out4 = nullptr;
    double *csum = nullptr;                  // chunk sums of the line reductions
    // imaginary-time convergence on the device: [0] stop word (int), [8] steps done (int64_t)
    unsigned char *istate = nullptr;
    double *eprev = nullptr;                 // [batch] energies of the last check
    const int *cur_stop = nullptr;           // set while gpe_step_imag runs: kernels check it
    double *ones = nullptr;                 // [batch] of 1.0 (resets the renormalisation factors)
    int *err = nullptr;
    int64_t lines_cap = 0;
    double *pin = nullptr;   // pinned host staging
    size_t pin_len = 0;
    void *work[4] = {};
    double *hist = nullptr, *spec_out = nullptr;
    int hist_blocks = 0;
    int64_t nshells = 0;
    void *host_buf = nullptr;    // device copy for gpe_step_real_host
    // slab pipeline of gpe_step_real_host: a copy stream and one event per slab and direction
    cudaStream_t copy_st = nullptr;
    cudaEvent_t slab_ev[2][16] = {};
    std::vector<void *> allocs;
    // launch context for batches of separately allocated instances (serve.cu):
    // when cur_count > 0, launches cover cur_count instances found through
    // cur_ptrs (device array of base pointers) using table slots cur_slots
    void *const *cur_ptrs = nullptr;
    const int *cur_slots = nullptr;
    int64_t cur_count = 0;
    std::vector<double> gamma_host;   // [batch][3], host copy of the trap parameters
    // tracing
    bool tracing = false;
    struct Rec { std::string kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
    std::vector<std::string> kinds;
    std::map<std::string, std::pair<int64_t, double>> totals;
    // tensor maps of the swept array for the strided axes, rebuilt when the
    // array, axis or instance count changes
    struct Tmap { const void *ptr = nullptr; int64_t batch = 0; int lines = 0; bool ok = false; CUtensorMap map; };
    Tmap tmaps[3];
    bool use_tma[3] = {true, true, true};   // copy-engine staging per axis (strided axes only)
    int tile_var[3] = {0, 0, 0};            // tile shape per axis
    int tx_extra = 0;                       // GPE_OPT_TEST_STALL_COPIES
    bool generic_passes = false;            // GPE_OPT_GENERIC_PASSES
    bool line_cluster = true;               // GPE_OPT_LINE_CLUSTER
    bool no_dither = false;                 // GPE_OPT_NO_DITHER
    // trap tables of one time level (gpe_step_real_trap), allocated on first use
    void *sched[3] = {nullptr, nullptr, nullptr};
    void *sched_last = nullptr;
    double *dtab = nullptr;                 // dither angles and offsets per step (resident kernel)
};

static gpe_status check_err(gpe_plan *p);

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// instances covered by the launches of the current call
static int64_t active_count(const gpe_plan *p) { return p->cur_count > 0 ? p->cur_count : p->batch; }

static int ilog2_64(int64_t v)
{
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}
static bool pow2(int64_t v) { return v >= 1 && (v & (v - 1)) == 0; }

static gpe_status dalloc(gpe_plan *p, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return GPE_OK;
    GPE_CUDA(cudaMalloc(ptr, bytes));
    p->allocs.push_back(*ptr);
    return GPE_OK;
}

// upload a double-precision table rounded to the bulk precision
static gpe_status upload_real(gpe_plan *p, void **dst, const std::vector<double> &v)
{
    GPE_TRY(dalloc(p, dst, v.size() * p->rsize));
    if (p->prec == GPE_C64) {
        std::vector<float> f(v.begin(), v.end());
        GPE_CUDA(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        GPE_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return GPE_OK;
}
// v holds interleaved (re, im) of unit factors.  complex128: stored as is;
// complex64: each value w becomes (hi, lo) = (fl(w), fl(w - fl(w))) so that
// kernels can apply it without a per-application modulus error.
static gpe_status upload_cplx(gpe_plan *p, void **dst, const std::vector<double> &v)
{
    if (p->prec != GPE_C64) return upload_real(p, dst, v);
    GPE_TRY(dalloc(p, dst, v.size() * 2 * sizeof(float)));
    std::vector<float> f(v.size() * 2);
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        const float hx = (float)v[i], hy = (float)v[i + 1];
        f[2 * i + 0] = hx;
        f[2 * i + 1] = hy;
        f[2 * i + 2] = (float)(v[i] - (double)hx);
        f[2 * i + 3] = (float)(v[i + 1] - (double)hy);
    }
    GPE_CUDA(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    return GPE_OK;
}

static void destroy(gpe_plan *p)
{
    if (!p) return;
    for (auto &r : p->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : p->event_pool) cudaEventDestroy(e);
    for (void *a : p->allocs) cudaFree(a);
    if (p->pin) cudaFreeHost(p->pin);
    for (auto &row : p->slab_ev)
        for (auto e : row)
            if (e) cudaEventDestroy(e);
    if (p->copy_st) cudaStreamDestroy(p->copy_st);
    delete p;
}

// Trap tables of one instance on axis a (V_a = gamma^2 x^2 / 2, th = V_a dt):
// vh = exp(-i th/2) - 1, vf = exp(-i th) - 1 (interleaved re, im), vi = exp(-th/2).
static void trap_tables_host(const gpe_plan *p, int a, double gamma, double *vh, double *vf, double *vi)
{
    const int64_t na = p->n[a];
    for (int64_t j = 0; j < na; ++j) {
        const double x = p->lo[a] + (double)j * p->h[a];
        const double th = 0.5 * gamma * gamma * x * x * p->dt;
        vh[2 * j] = -2.0 * sin(0.25 * th) * sin(0.25 * th);
        vh[2 * j + 1] = -sin(0.5 * th);
        vf[2 * j] = -2.0 * sin(0.5 * th) * sin(0.5 * th);
        vf[2 * j + 1] = -sin(th);
        vi[j] = exp(-0.5 * th);
    }
}

// complex table values (re, im) in the device format of the plan's precision
static void pack_cplx(const gpe_plan *p, const std::vector<double> &v, std::vector<unsigned char> &out)
{
    if (p->prec != GPE_C64) {
        out.resize(v.size() * sizeof(double));
        memcpy(out.data(), v.data(), out.size());
        return;
    }
    std::vector<float> f(v.size() * 2);
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        const float hx = (float)v[i], hy = (float)v[i + 1];
        f[2 * i + 0] = hx;
        f[2 * i + 1] = hy;
        f[2 * i + 2] = (float)(v[i] - (double)hx);
        f[2 * i + 3] = (float)(v[i + 1] - (double)hy);
    }
    out.resize(f.size() * sizeof(float));
    memcpy(out.data(), f.data(), out.size());
}

extern "C" gpe_status gpe_plan_create(const gpe_plan_desc *d, void *cuda_stream, gpe_plan **out)
{
    if (!d || !out) return fail(GPE_EINVAL, "gpe_plan_create: NULL argument");
    *out = nullptr;
    if (d->ndim < 1 || d->ndim > 3) return fail(GPE_EUNSUPPORTED, "ndim must be 1, 2 or 3");
    if (d->prec != GPE_C64 && d->prec != GPE_C128) return fail(GPE_EINVAL, "prec must be GPE_C64 or GPE_C128");
    if (d->batch < 1) return fail(GPE_EINVAL, "batch must be >= 1");
    if (!isfinite(d->dt) || !isfinite(d->g)) return fail(GPE_EINVAL, "dt and g must be finite");
    for (int a = 0; a < d->ndim; ++a) {
        if (!pow2(d->n[a]) || d->n[a] < 2 || d->n[a] > 4096)
            return fail(GPE_EUNSUPPORTED, "each n[a] must be a power of two in [2, 4096]");
        if (!(d->len[a] > 0.0) || !isfinite(d->len[a]) || !isfinite(d->lo[a]))
            return fail(GPE_EINVAL, "len[a] must be positive and lo[a] finite");
    }
    gpe_plan *p = new gpe_plan();
    p->ndim = d->ndim;
    p->batch = d->batch;
    p->prec = d->prec;
    p->csize = d->prec == GPE_C64 ? 8 : 16;
    p->rsize = d->prec == GPE_C64 ? 4 : 8;
    p->dt = d->dt;
    p->st = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        destroy(p);
        return fail(GPE_ECUDA, "cudaGetDevice failed");
    }
    for (int a = 0; a < 3; ++a) {
        p->n[a] = a < d->ndim ? d->n[a] : 1;
        p->lo[a] = a < d->ndim ? d->lo[a] : 0.0;
        p->len[a] = a < d->ndim ? d->len[a] : 1.0;
        p->h[a] = a < d->ndim ? d->len[a] / (double)d->n[a] : 0.0;
        p->kf[a] = a < d->ndim ? 2.0 * M_PI / d->len[a] : 0.0;
        p->N *= p->n[a];
    }
    p->dv = 1.0;
    for (int a = 0; a < d->ndim; ++a) p->dv *= p->h[a];

    const int64_t B = p->batch;
    if (d->V_host) {
        bool ok = !d->gamma_each;
        for (int a = 0; a < d->ndim; ++a) ok = ok && d->gamma[a] == 0.0;
        for (int64_t i = 0; ok && i < p->N; ++i) ok = isfinite(d->V_host[i]);
        if (!ok) {
            destroy(p);
            return fail(GPE_EINVAL, "V_host needs finite values and gamma = 0, gamma_each = NULL");
        }
    }
    std::vector<double> gs(B), gam(3 * B, 0.0);
    for (int64_t b = 0; b < B; ++b) {
        gs[b] = d->g_each ? d->g_each[b] : d->g;
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            if (a < d->ndim) v = d->gamma_each ? d->gamma_each[3 * b + a] : d->gamma[a];
            if (!isfinite(v) || !isfinite(gs[b])) {
                destroy(p);
                return fail(GPE_EINVAL, "g and gamma must be finite");
            }
            gam[3 * b + a] = v;
            if (v != 0.0) p->trap[a] = true;
        }
    }
    gpe_status s = GPE_OK;
#define PLAN_TRY(expr)            \
    do {                          \
        s = (expr);               \
        if (s != GPE_OK) {        \
            destroy(p);           \
            return s;             \
        }                         \
    } while (0)
    for (int a = 0; a < d->ndim; ++a) {
        const int64_t na = p->n[a];
        std::vector<double> tw(2 * na), kt(2 * na), ki(na);
        for (int64_t t = 0; t < na; ++t) {
            const double ang = 2.0 * M_PI * (double)t / (double)na;
            tw[2 * t] = cos(ang);
            tw[2 * t + 1] = -sin(ang);
            const int64_t m = t < na / 2 ? t : t - na;
            const double k = p->kf[a] * (double)m;
            const double th = 0.5 * k * k * p->dt;
            // offset exp(-i th) - 1 = (-2 sin^2(th/2), -sin th)
            kt[2 * t] = -2.0 * sin(0.5 * th) * sin(0.5 * th);
            kt[2 * t + 1] = -sin(th);
            ki[t] = exp(-th) / (double)na;
        }
        PLAN_TRY(upload_cplx(p, &p->tw[a], tw));
        PLAN_TRY(upload_cplx(p, &p->kt[a], kt));
        PLAN_TRY(upload_real(p, &p->ki[a], ki));
        if (p->trap[a]) {
            std::vector<double> vh(2 * na * B), vf(2 * na * B), vi(na * B);
            for (int64_t b = 0; b < B; ++b)
                trap_tables_host(p, a, gam[3 * b + a], &vh[2 * b * na], &vf[2 * b * na], &vi[b * na]);
            PLAN_TRY(upload_cplx(p, &p->vh[a], vh));
            PLAN_TRY(upload_cplx(p, &p->vf[a], vf));
            PLAN_TRY(upload_real(p, &p->vi[a], vi));
        }
    }
    if (d->V_host) {
        // the sampled values, and for 1D the same potential as trap tables of
        // the on-chip kernel (exact: in 1D a sampled V is a per-axis table)
        PLAN_TRY(upload_real(p, &p->vsamp, std::vector<double>(d->V_host, d->V_host + p->N)));
        if (d->ndim == 1) {
            const int64_t na = p->n[0];
            std::vector<double> vh(2 * na * B), vf(2 * na * B), vi(na * B);
            for (int64_t b = 0; b < B; ++b)
                for (int64_t j = 0; j < na; ++j) {
                    const double th = d->V_host[j] * p->dt;
                    vh[2 * (b * na + j)] = -2.0 * sin(0.25 * th) * sin(0.25 * th);
                    vh[2 * (b * na + j) + 1] = -sin(0.5 * th);
                    vf[2 * (b * na + j)] = -2.0 * sin(0.5 * th) * sin(0.5 * th);
                    vf[2 * (b * na + j) + 1] = -sin(th);
                    vi[b * na + j] = exp(-0.5 * th);
                }
            PLAN_TRY(upload_cplx(p, &p->vh[0], vh));
            PLAN_TRY(upload_cplx(p, &p->vf[0], vf));
            PLAN_TRY(upload_real(p, &p->vi[0], vi));
            p->trap[0] = true;
        }
    }
    // per-instance parameters and reduction buffers (always double precision)
    int64_t maxlines = 0;
    for (int a = 0; a < d->ndim; ++a) maxlines = std::max<int64_t>(maxlines, p->N / p->n[a]);
    p->lines_cap = maxlines * B;
    PLAN_TRY(dalloc(p, (void **)&p->g_dev, sizeof(double) * B));
    PLAN_TRY(dalloc(p, (void **)&p->gamma_dev, sizeof(double) * 3 * B));
    PLAN_TRY(dalloc(p, (void **)&p->scale, sizeof(double) * B));
    PLAN_TRY(dalloc(p, (void **)&p->partials, sizeof(double) * NQ * p->lines_cap));
    PLAN_TRY(dalloc(p, (void **)&p->sums, sizeof(double) * NQ * B));
    {
        int64_t nch = 1;
        for (int a = 0; a < d->ndim; ++a) nch = std::max(nch, reduce_chunks(p->N / p->n[a]));
        PLAN_TRY(dalloc(p, (void **)&p->csum, sizeof(double) * NQ * B * nch));
    }
    PLAN_TRY(dalloc(p, (void **)&p->istate, 16));
    PLAN_TRY(dalloc(p, (void **)&p->eprev, sizeof(double) * B));
    PLAN_TRY(dalloc(p, (void **)&p->out6, sizeof(double) * 6 * B));
    PLAN_TRY(dalloc(p, (void **)&p->out4, sizeof(double) * 4 * B));
    PLAN_TRY(dalloc(p, (void **)&p->err, sizeof(int)));
    PLAN_TRY(dalloc(p, (void **)&p->ones, sizeof(double) * B));
#undef PLAN_TRY
    p->gamma_host = gam;
    {
        std::vector<double> one(B, 1.0);
        if (cudaMemcpy(p->ones, one.data(), sizeof(double) * B, cudaMemcpyHostToDevice) != cudaSuccess) {
            destroy(p);
            return fail(GPE_ECUDA, "uploading plan parameters failed");
        }
    }
    if (cudaMemcpy(p->g_dev, gs.data(), sizeof(double) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->gamma_dev, gam.data(), sizeof(double) * 3 * B, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess) {
        destroy(p);
        return fail(GPE_ECUDA, "uploading plan parameters failed");
    }
    p->pin_len = (size_t)B * 6 + 64;
    if (cudaMallocHost((void **)&p->pin, sizeof(double) * p->pin_len) != cudaSuccess) {
        p->pin = nullptr;
        destroy(p);
        return fail(GPE_ENOMEM, "pinned host staging allocation failed");
    }
    *out = p;
    return GPE_OK;
}

extern "C" gpe_status gpe_plan_destroy(gpe_plan *p)
{
    if (!p) return fail(GPE_EINVAL, "gpe_plan_destroy: NULL plan");
    DeviceGuard dg(p->device);
    if (p->st) cudaStreamSynchronize(p->st);
    else cudaDeviceSynchronize();
    destroy(p);
    return GPE_OK;
}

// ------------------------------------------------------------------ tracing
static cudaEvent_t pool_event(gpe_plan *p)
{
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Bracket one launch with events when tracing is on.
struct TraceScope {
    gpe_plan *p;
    std::string kind;
    cudaEvent_t a = nullptr;
    TraceScope(gpe_plan *p_, std::string k) : p(p_), kind(std::move(k))
    {
        if (p->tracing && (a = pool_event(p))) cudaEventRecord(a, p->st);
    }
    ~TraceScope()
    {
        if (!a) return;
        cudaEvent_t b = pool_event(p);
        if (!b) { p->event_pool.push_back(a); return; }
        cudaEventRecord(b, p->st);
        p->recs.push_back({kind, a, b});
    }
};

static gpe_status trace_flush(gpe_plan *p)
{
    if (p->recs.empty()) return GPE_OK;
    GPE_CUDA(cudaStreamSynchronize(p->st));
    for (auto &r : p->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto it = p->totals.find(r.kind);
        if (it == p->totals.end()) {
            p->kinds.push_back(r.kind);
            p->totals[r.kind] = {1, (double)ms};
        } else {
            it->second.first += 1;
            it->second.second += ms;
        }
        p->event_pool.push_back(r.a);
        p->event_pool.push_back(r.b);
    }
    p->recs.clear();
    return GPE_OK;
}

extern "C" gpe_status gpe_trace_enable(gpe_plan *p, int enable)
{
    if (!p) return fail(GPE_EINVAL, "NULL plan");
    DeviceGuard dg(p->device);
    GPE_TRY(trace_flush(p));
    p->kinds.clear();
    p->totals.clear();
    p->tracing = enable != 0;
    return GPE_OK;
}

extern "C" int gpe_trace_count(gpe_plan *p)
{
    if (!p) return -1;
    DeviceGuard dg(p->device);
    if (trace_flush(p) != GPE_OK) return -1;
    return (int)p->kinds.size();
}

extern "C" gpe_status gpe_trace_read(gpe_plan *p, int i, char *name, size_t name_len, int64_t *launches,
                                     double *total_ms)
{
    if (!p) return fail(GPE_EINVAL, "NULL plan");
    DeviceGuard dg(p->device);
    GPE_TRY(trace_flush(p));
    if (i < 0 || i >= (int)p->kinds.size()) return fail(GPE_EINVAL, "trace index out of range");
    const std::string &k = p->kinds[i];
    if (name && name_len) {
        size_t m = std::min(name_len - 1, k.size());
        memcpy(name, k.data(), m);
        name[m] = 0;
    }
    if (launches) *launches = p->totals[k].first;
    if (total_ms) *total_ms = p->totals[k].second;
    return GPE_OK;
}

static const char *op_tag(int op)
{
    switch (op) {
    case OP_NREAL: return "NR";
    case OP_NIMAG: return "NI";
    case OP_KREAL: return "KR";
    case OP_KIMAG: return "KI";
    case OP_SCALE_NIMAG: return "S-NI";
    case OP_SCALE: return "S";
    default: return "";
    }
}

static std::string pass_kind(const PassArgs &a)
{
    std::string s = std::string(1, "xyz"[a.axis]) + std::to_string(a.nax) + ":";
    if (a.red == RED_DIAG_X || a.red == RED_DIAG_K || a.red == RED_DIAG_XM) return s + "diag";
    std::vector<std::string> parts;
    auto add = [&](const char *t) { if (*t) parts.push_back(t); };
    add(op_tag(a.op_pre));
    add(a.fft1 < 0 ? "F" : a.fft1 > 0 ? "I" : "");
    add(op_tag(a.op_mid));
    add(a.fft2 < 0 ? "F" : a.fft2 > 0 ? "I" : "");
    add(op_tag(a.op_post));
    if (a.red == RED_NORM) parts.push_back("red");
    for (size_t i = 0; i < parts.size(); ++i) s += (i ? "-" : "") + parts[i];
    return s;
}

// ------------------------------------------------------------------ pass setup
// Geometry of a sweep along `axis` over `batch` instances starting at src/dst.
static PassArgs make_pass(const gpe_plan *p, int axis, const void *src, void *dst, int64_t batch)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    const int64_t n0 = p->n[0], n1 = p->n[1];
    a.src = src;
    a.dst = dst;
    a.nax = (int)p->n[axis];
    a.axis = axis;
    const int64_t lpi = p->N / p->n[axis];
    a.lg_lpi = ilog2_64(lpi);
    a.inst_stride = p->N;
    int o0 = -1, o1 = -1;
    if (axis == 0) {
        a.lg_A = 0;
        a.Sb = n0;
        a.estride = 1;
        o0 = 1;
        o1 = 2;
    } else if (axis == 1) {
        a.lg_A = ilog2_64(n0);
        a.Sb = n0 * n1;
        a.estride = n0;
        o0 = 0;
        o1 = 2;
    } else {
        a.lg_A = ilog2_64(n0 * n1);
        a.Sb = p->N;
        a.estride = n0 * n1;
        o0 = 0;
        o1 = 1;
    }
    a.o0n = (int)p->n[o0];
    a.o1n = (int)p->n[o1];
    a.lg_o0 = ilog2_64(p->n[o0]);
    a.lines_total = batch * lpi;
    const int L = pass_lines_per_tile(p->prec, axis == 0, a.nax, p->tile_var[axis]);
    a.ntiles = (a.lines_total + L - 1) / L;
    a.tw = p->tw[axis];
    const bool h0 = o0 < p->ndim, h1 = o1 < p->ndim;
    a.kt_ax = p->kt[axis];
    a.kt_o0 = h0 ? p->kt[o0] : nullptr;
    a.kt_o1 = h1 ? p->kt[o1] : nullptr;
    a.ki_ax = p->ki[axis];
    a.ki_o0 = h0 ? p->ki[o0] : nullptr;
    a.ki_o1 = h1 ? p->ki[o1] : nullptr;
    a.vi_ax = p->vi[axis];
    a.vi_o0 = h0 ? p->vi[o0] : nullptr;
    a.vi_o1 = h1 ? p->vi[o1] : nullptr;
    a.vsamp = p->ndim >= 2 ? p->vsamp : nullptr;
    a.vsamp_diag = p->vsamp;
    a.g = p->g_dev;
    a.inv_n = 1.0 / (double)p->N;
    // states of up to 64 MiB (1024^2 complex64 is 8 MiB): every sweep is one
    // short wave of CTAs, and the next kernel's launch may start with it
    // (1024^2 complex64 step 27.1 -> 25.5 us); larger states trigger it at
    // the end of each CTA (512^3 complex64: 2.39 ms/step with the early
    // trigger, 2.15 with the late one, 2.16 without dependent launch)
    a.pdl_early = (double)p->N * (double)batch * (p->prec == GPE_C64 ? 8.0 : 16.0) <= 64.0 * 1048576.0;
    a.stop = p->cur_stop;
    a.scale = p->scale;
    a.partials = p->partials;
    a.lines_cap = p->lines_cap;
    a.gamma = p->gamma_dev;
    for (int i = 0; i < 3; ++i) {
        a.lo[i] = i < p->ndim ? p->lo[i] : 0.0;
        a.h[i] = i < p->ndim ? p->h[i] : 0.0;
        a.kf[i] = p->kf[i];
    }
    a.fft1 = a.fft2 = 0;
    a.op_pre = a.op_mid = a.op_post = OP_NONE;
    a.red = RED_NONE;
    if (p->cur_count > 0 && src == p->cur_ptrs) {
        a.inst_ptr = p->cur_ptrs;
        a.slot_of = p->cur_slots;
        a.src = a.dst = nullptr;
    }
    return a;
}

// select the real-time trap tables for a nonlinear substep of length c*dt (c = 1/2 or 1)
static void set_nreal(const gpe_plan *p, PassArgs &a, bool full)
{
    void *const *vt = full ? p->vf : p->vh;
    const int axis = a.axis;
    const int o0 = axis == 0 ? 1 : 0, o1 = axis == 2 ? 1 : 2;
    a.vt_ax = vt[axis];
    a.vt_o0 = o0 < p->ndim ? vt[o0] : nullptr;
    a.vt_o1 = o1 < p->ndim ? vt[o1] : nullptr;
    a.nl_c = full ? p->dt : 0.5 * p->dt;
}

// ------------------------------------------------------------------ tensor maps
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library links no driver stub)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

// Tensor map of `batch` back-to-back instances at ptr, viewed as the 4D array
// [batch][n2][n1][n0] of 8-byte elements (complex128 points are two of them
// along n0), with a box of L lines by `box` points along `axis` (1 or 2).
static bool make_tmap(const gpe_plan *p, int axis, const void *ptr, int64_t batch, int L, int box, CUtensorMap *m)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const int64_t w = (int64_t)(p->csize / 8);        // 8-byte elements per point
    cuuint64_t dim[4] = {(cuuint64_t)(p->n[0] * w), (cuuint64_t)p->n[1], (cuuint64_t)p->n[2], (cuuint64_t)batch};
    cuuint64_t stride[3] = {(cuuint64_t)(p->n[0] * p->csize), (cuuint64_t)(p->n[0] * p->n[1] * p->csize),
                            (cuuint64_t)(p->N * p->csize)};
    cuuint32_t boxd[4] = {(cuuint32_t)(L * w), axis == 1 ? (cuuint32_t)box : 1u, axis == 2 ? (cuuint32_t)box : 1u, 1u};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<void *>(ptr), dim, stride, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static gpe_status run(gpe_plan *p, const PassArgs &a_in)
{
    PassArgs a = a_in;
    a.err = p->err;
    a.generic = p->generic_passes ? 1 : 0;
    const CUtensorMap *tm = nullptr;
    // strided sweeps over one array of back-to-back instances, with whole
    // tiles of consecutive x lines, take the copy-engine staging
    const int var = p->tile_var[a.axis];
    if (p->use_tma[a.axis] && a.axis >= 1 && a.src && !a.inst_ptr && (a.dst == nullptr || a.dst == a.src)) {
        const int L = pass_lines_per_tile(p->prec, false, a.nax, var);
        const int box = a.nax < 256 ? a.nax : 256;
        const int64_t lpi = p->N / p->n[a.axis];
        const int64_t batch = (a.lines_total + lpi - 1) / lpi;   // instances the sweep reaches (a slab: its own)
        if (p->n[0] % L == 0 && ((uintptr_t)a.src) % 16 == 0) {
            gpe_plan::Tmap &c = p->tmaps[a.axis];
            if (!c.ok || c.ptr != a.src || c.batch != batch || c.lines != L) {
                c.ok = make_tmap(p, a.axis, a.src, batch, L, box, &c.map);
                c.ptr = a.src;
                c.batch = batch;
                c.lines = L;
            }
            if (c.ok) {
                tm = &c.map;
                a.tma_box = box;
                a.tma_chunks = a.nax / box;
                a.tx_extra = p->tx_extra;
            }
        }
    }
    TraceScope ts(p, pass_kind(a));
    cudaError_t e = launch_pass(p->prec, a.axis == 0, a, p->st, tm, var);
    if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("pass launch: ") + cudaGetErrorString(e));
    return GPE_OK;
}

static gpe_status check_psi(const gpe_plan *p, const void *psi)
{
    if (!p) return fail(GPE_EINVAL, "NULL plan");
    if (!psi) return fail(GPE_EINVAL, "NULL psi");
    if (((uintptr_t)psi) % 16 != 0) return fail(GPE_EINVAL, "psi must be 16-byte aligned");
    return GPE_OK;
}

// ------------------------------------------------------------------ real time
// Phase dither of the complex64 real-time step.  The kinetic substep of step
// s also multiplies by exp(-i phi_s) and the nonlinear substep that follows
// it in the same step by exp(+i phi_s); in exact arithmetic the two cancel
// (a global phase, applied and removed within the step), so the method is
// unchanged.  Without it the slowly turning low-k modes, which hold most of
// the norm, are rounded in nearly the same way step after step: their
// rounding errors do not average out and the norm drifts (about 1e-9 per step
// on the 2D turbulence workload).  A global turn of up to 0.01 rad moves every
// value by ~1e5 units in the last place, so successive roundings decorrelate
// and the norm error becomes a random walk.  phi_s is a fixed low-discrepancy
// sequence of the step index in the call, so results are reproducible.
static double dither_angle(int64_t s)
{
    const double g = 0.6180339887498948482;      // golden-ratio sequence in [-0.01, 0.01), period 2^16
    const double f = (double)(s & (GPE_DITHER_PERIOD - 1)) * g + 0.5;
    return 0.02 * (f - floor(f)) - 0.01;
}
static void set_dither(PassArgs &k, double phi)
{
    // offset exp(-i phi) - 1 = (-2 sin^2(phi/2), -sin phi) as hi + lo floats
    const double sh = sin(0.5 * phi);
    const double wx = -2.0 * sh * sh, wy = -sin(phi);
    const float hx = (float)wx, hy = (float)wy;
    k.dither = 1;
    k.dk[0] = hx;
    k.dk[1] = hy;
    k.dk[2] = (float)(wx - (double)hx);
    k.dk[3] = (float)(wy - (double)hy);
}

// Trap tables of time level `lev` of a schedule (rows of three gamma) for a
// nonlinear substep of length c dt, written into dst[a] for every instance.
static gpe_status trap_level(gpe_plan *p, void *const *dst, const double *gamma_t, int64_t lev, double c)
{
    double gm[3] = {0, 0, 0};
    for (int a = 0; a < p->ndim; ++a) gm[a] = gamma_t[3 * lev + a];
    cudaError_t e = launch_trap_level(p->prec == GPE_C64 ? 0 : 1, dst, p->ndim, p->n, p->lo, p->h, gm, c * p->dt,
                                      p->batch, p->st);
    if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("trap tables: ") + cudaGetErrorString(e));
    return GPE_OK;
}
static void use_sched(const gpe_plan *p, PassArgs &a)
{
    const int axis = a.axis;
    const int o0 = axis == 0 ? 1 : 0, o1 = axis == 2 ? 1 : 2;
    a.vt_ax = p->sched[axis];
    a.vt_o0 = o0 < p->ndim ? p->sched[o0] : nullptr;
    a.vt_o1 = o1 < p->ndim ? p->sched[o1] : nullptr;
}

// nsteps real-time steps; with gamma_t (nsteps + 1 rows of three trap
// frequencies) the harmonic trap follows that schedule instead of the plan's
// static trap: the nonlinear half-steps next to time level n use gamma_t row n.
static gpe_status step_real_dev(gpe_plan *p, void *psi, int64_t nsteps, const double *gamma_t = nullptr)
{
    if (nsteps == 0) return GPE_OK;
    const int64_t B = active_count(p);
    if (p->ndim == 1 && gamma_t) {
        // one on-chip launch per step, with the trap of both of its time levels
        for (int64_t s = 0; s < nsteps; ++s) {
            GPE_TRY(trap_level(p, p->sched, gamma_t, s, 0.5));
            GPE_TRY(trap_level(p, &p->sched_last, gamma_t, s + 1, 0.5));
            Line1DArgs l;
            memset(&l, 0, sizeof(l));
            l.psi = psi;
            l.batch = B;
            l.n = (int)p->n[0];
            l.nsteps = 1;
            l.tw = p->tw[0];
            l.kt = p->kt[0];
            l.vh = p->sched[0];
            l.vh_last = p->sched_last;
            l.g = p->g_dev;
            l.dt = p->dt;
            l.err = p->err;
            l.cluster = p->line_cluster ? 1 : 0;
            l.tx_extra = p->tx_extra;
            if (p->cur_count > 0) {
                l.inst_ptr = p->cur_ptrs;
                l.slot_of = p->cur_slots;
            }
            TraceScope ts(p, "line1d" + std::to_string(l.n) + ":real");
            cudaError_t e = launch_line1d(p->prec, l, p->st);
            if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("1D launch: ") + cudaGetErrorString(e));
        }
        return GPE_OK;
    }
    if (p->ndim == 1) {
        const int64_t chunk = 1 << 16;
        for (int64_t done = 0; done < nsteps; done += chunk) {
            Line1DArgs l;
            memset(&l, 0, sizeof(l));
            l.psi = psi;
            l.batch = B;
            l.n = (int)p->n[0];
            l.nsteps = std::min(chunk, nsteps - done);
            l.imag = 0;
            l.tw = p->tw[0];
            l.kt = p->kt[0];
            l.vh = p->vh[0];
            l.vf = p->vf[0];
            l.g = p->g_dev;
            l.dt = p->dt;
            l.err = p->err;
            l.cluster = p->line_cluster ? 1 : 0;
            l.tx_extra = p->tx_extra;
            if (p->cur_count > 0) {
                l.inst_ptr = p->cur_ptrs;
                l.slot_of = p->cur_slots;
            }
            TraceScope ts(p, "line1d" + std::to_string(l.n) + ":real");
            cudaError_t e = launch_line1d(p->prec, l, p->st);
            if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("1D launch: ") + cudaGetErrorString(e));
        }
        return GPE_OK;
    }
    // prologue: first nonlinear half-step and forward transforms of all but the last axis
    PassArgs x0 = make_pass(p, 0, psi, psi, B);
    x0.op_pre = OP_NREAL;
    set_nreal(p, x0, false);
    if (gamma_t) {
        GPE_TRY(trap_level(p, p->sched, gamma_t, 0, 0.5));
        use_sched(p, x0);
    }
    x0.fft1 = -1;
    GPE_TRY(run(p, x0));
    if (p->ndim == 3) {
        PassArgs y = make_pass(p, 1, psi, psi, B);
        y.fft1 = -1;
        GPE_TRY(run(p, y));
    }
    const int piv = p->ndim - 1;
    const bool dither = p->prec == GPE_C64 && !p->no_dither;
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        PassArgs k = make_pass(p, piv, psi, psi, B);
        k.fft1 = -1;
        k.op_mid = OP_KREAL;
        k.fft2 = +1;
        const double phi = dither ? dither_angle(s) : 0.0;
        if (dither) set_dither(k, phi);
        GPE_TRY(run(p, k));
        if (p->ndim == 3) {
            PassArgs y = make_pass(p, 1, psi, psi, B);
            y.fft1 = +1;
            GPE_TRY(run(p, y));
        }
        PassArgs x = make_pass(p, 0, psi, psi, B);
        x.fft1 = +1;
        x.op_mid = OP_NREAL;
        set_nreal(p, x, !last);
        if (gamma_t) {
            GPE_TRY(trap_level(p, p->sched, gamma_t, s + 1, last ? 0.5 : 1.0));
            use_sched(p, x);
        }
        x.dphi = phi;
        x.fft2 = last ? 0 : -1;
        GPE_TRY(run(p, x));
        if (p->ndim == 3 && !last) {
            PassArgs y = make_pass(p, 1, psi, psi, B);
            y.fft1 = -1;
            GPE_TRY(run(p, y));
        }
    }
    return GPE_OK;
}

extern "C" gpe_status gpe_step_real_trap(gpe_plan *p, void *psi, int64_t nsteps, const double *gamma_host)
{
    GPE_TRY(check_psi(p, psi));
    if (nsteps < 0) return fail(GPE_EINVAL, "nsteps must be >= 0");
    if (!gamma_host) return fail(GPE_EINVAL, "gamma_host is NULL");
    if (p->vsamp) return fail(GPE_EUNSUPPORTED, "a trap schedule replaces the potential: plans with V_host have none");
    for (int64_t i = 0; i < 3 * (nsteps + 1); ++i)
        if (!isfinite(gamma_host[i])) return fail(GPE_EINVAL, "trap frequencies must be finite");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(GPE_ECUDA, "cannot select the plan's device");
    const size_t ce = p->prec == GPE_C64 ? sizeof(float4) : sizeof(double2);
    for (int a = 0; a < p->ndim; ++a)
        if (!p->sched[a]) GPE_TRY(dalloc(p, &p->sched[a], ce * (size_t)p->n[a] * (size_t)p->batch));
    if (p->ndim == 1 && !p->sched_last) GPE_TRY(dalloc(p, &p->sched_last, ce * (size_t)p->n[0] * (size_t)p->batch));
    return step_real_dev(p, psi, nsteps, gamma_host);
}

extern "C" gpe_status gpe_step_real(gpe_plan *p, void *psi, int64_t nsteps)
{
    GPE_TRY(check_psi(p, psi));
    if (nsteps < 0) return fail(GPE_EINVAL, "nsteps must be >= 0");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(GPE_ECUDA, "cannot select the plan's device");
    return step_real_dev(p, psi, nsteps);
}

// Restrict a sweep to lines [first, first + count) of its axis (a slab of the
// grid: whole planes of the slowest axis, so the lines are consecutive and
// every tile starts on a tile boundary).
static void restrict_lines(const gpe_plan *p, PassArgs &a, int axis, int64_t first, int64_t count)
{
    const int L = pass_lines_per_tile(p->prec, axis == 0, (int)p->n[axis], p->tile_var[axis]);
    a.line0 = first;
    a.lines_total = first + count;
    a.ntiles = (count + L - 1) / L;
}

// gpe_step_real_host for one instance of at least 64 MiB in pinned host
// memory: the state moves in slabs of whole planes of the slowest axis, and
// the sweeps that stay inside a slab (the call's first nonlinear half-step
// with the x transform, and the forward y transform in 3D; at the end the
// inverse y transform and the last x sweep) run on each slab as soon as it has
// arrived / before it leaves, on the plan stream, while the copy stream moves
// the other slabs.  Every line is computed as in step_real_dev.
static gpe_status step_real_host_slabs_enqueue(gpe_plan *p, unsigned char *host, int64_t nsteps, int S);
static gpe_status step_real_host_slabs(gpe_plan *p, unsigned char *host, int64_t nsteps, int S)
{
    const gpe_status st = step_real_host_slabs_enqueue(p, host, nsteps, S);
    if (st != GPE_OK) {
        // no copy into or out of the caller's buffer may outlive the call
        if (p->copy_st) cudaStreamSynchronize(p->copy_st);
        cudaStreamSynchronize(p->st);
        return st;
    }
    GPE_CUDA(cudaStreamSynchronize(p->copy_st));
    return check_err(p);
}
static gpe_status step_real_host_slabs_enqueue(gpe_plan *p, unsigned char *host, int64_t nsteps, int S)
{
    const int d = p->ndim;
    const int64_t nslow = p->n[d - 1];
    const int64_t planes = nslow / S;
    const size_t plane_bytes = (size_t)(p->N / nslow) * p->csize;
    unsigned char *dev = static_cast<unsigned char *>(p->host_buf);
    if (!p->copy_st) GPE_CUDA(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking));
    for (int k = 0; k < S; ++k)
        for (int dir = 0; dir < 2; ++dir)
            if (!p->slab_ev[dir][k]) GPE_CUDA(cudaEventCreateWithFlags(&p->slab_ev[dir][k], cudaEventDisableTiming));
    // lines of a slab on the x axis (rows: all but x; the slowest axis slowest)
    // and, in 3D, on the y axis (x and z; z slowest)
    const int64_t rows_per_plane = p->N / nslow / p->n[0];
    const int64_t ylines_per_plane = d == 3 ? p->n[0] : 0;
    auto slab_pass = [&](PassArgs a, int axis, int k) -> gpe_status {
        const int64_t per = axis == 0 ? rows_per_plane : ylines_per_plane;
        restrict_lines(p, a, axis, (int64_t)k * planes * per, planes * per);
        return run(p, a);
    };
    // the plan stream must not start before earlier work on psi_host's device copy ends
    GPE_CUDA(cudaEventRecord(p->slab_ev[1][0], p->st));
    GPE_CUDA(cudaStreamWaitEvent(p->copy_st, p->slab_ev[1][0], 0));
    for (int k = 0; k < S; ++k) {
        const size_t off = (size_t)k * planes * plane_bytes, len = (size_t)planes * plane_bytes;
        GPE_CUDA(cudaMemcpyAsync(dev + off, host + off, len, cudaMemcpyHostToDevice, p->copy_st));
        GPE_CUDA(cudaEventRecord(p->slab_ev[0][k], p->copy_st));
    }
    if (nsteps == 0) {
        GPE_CUDA(cudaEventRecord(p->slab_ev[1][0], p->copy_st));
        GPE_CUDA(cudaStreamWaitEvent(p->st, p->slab_ev[1][0], 0));
    }
    // prologue per slab
    for (int k = 0; k < S && nsteps > 0; ++k) {
        GPE_CUDA(cudaStreamWaitEvent(p->st, p->slab_ev[0][k], 0));
        PassArgs x0 = make_pass(p, 0, dev, dev, 1);
        x0.op_pre = OP_NREAL;
        set_nreal(p, x0, false);
        x0.fft1 = -1;
        GPE_TRY(slab_pass(x0, 0, k));
        if (d == 3) {
            PassArgs y = make_pass(p, 1, dev, dev, 1);
            y.fft1 = -1;
            GPE_TRY(slab_pass(y, 1, k));
        }
    }
    const int piv = d - 1;
    const bool dither = p->prec == GPE_C64 && !p->no_dither;
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        PassArgs kp = make_pass(p, piv, dev, dev, 1);
        kp.fft1 = -1;
        kp.op_mid = OP_KREAL;
        kp.fft2 = +1;
        const double phi = dither ? dither_angle(s) : 0.0;
        if (dither) set_dither(kp, phi);
        GPE_TRY(run(p, kp));
        for (int k = 0; k < (last ? S : 1); ++k) {
            if (d == 3) {
                PassArgs y = make_pass(p, 1, dev, dev, 1);
                y.fft1 = +1;
                if (last) GPE_TRY(slab_pass(y, 1, k));
                else GPE_TRY(run(p, y));
            }
            PassArgs x = make_pass(p, 0, dev, dev, 1);
            x.fft1 = +1;
            x.op_mid = OP_NREAL;
            set_nreal(p, x, !last);
            x.dphi = phi;
            x.fft2 = last ? 0 : -1;
            if (last) {
                GPE_TRY(slab_pass(x, 0, k));
                // this slab is final: copy it out while the next ones finish
                GPE_CUDA(cudaEventRecord(p->slab_ev[1][k], p->st));
                GPE_CUDA(cudaStreamWaitEvent(p->copy_st, p->slab_ev[1][k], 0));
                const size_t off = (size_t)k * planes * plane_bytes, len = (size_t)planes * plane_bytes;
                GPE_CUDA(cudaMemcpyAsync(host + off, dev + off, len, cudaMemcpyDeviceToHost, p->copy_st));
            } else {
                GPE_TRY(run(p, x));
            }
        }
        if (d == 3 && !last) {
            PassArgs y = make_pass(p, 1, dev, dev, 1);
            y.fft1 = -1;
            GPE_TRY(run(p, y));
        }
    }
    if (nsteps == 0) {
        GPE_CUDA(cudaMemcpyAsync(host, dev, (size_t)nslow * plane_bytes, cudaMemcpyDeviceToHost, p->copy_st));
    }
    return GPE_OK;
}

extern "C" gpe_status gpe_step_real_host(gpe_plan *p, void *psi_host, int64_t nsteps)
{
    if (!p || !psi_host) return fail(GPE_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(GPE_EINVAL, "nsteps must be >= 0");
    DeviceGuard dg(p->device);
    const size_t bytes = (size_t)p->batch * (size_t)p->N * p->csize;
    if (!p->host_buf) GPE_TRY(dalloc(p, &p->host_buf, bytes));
    // pinned host memory of one large 2D/3D instance: pipelined slabs
    cudaPointerAttributes at;
    const bool pinned = cudaPointerGetAttributes(&at, psi_host) == cudaSuccess && at.type == cudaMemoryTypeHost;
    if (!pinned) cudaGetLastError();
    const int S = 8;
    if (pinned && p->ndim >= 2 && p->batch == 1 && p->cur_count == 0 && !p->vsamp && bytes >= (size_t)64 << 20 &&
        p->n[p->ndim - 1] % S == 0)
        return step_real_host_slabs(p, static_cast<unsigned char *>(psi_host), nsteps, S);
    GPE_CUDA(cudaMemcpyAsync(p->host_buf, psi_host, bytes, cudaMemcpyHostToDevice, p->st));
    GPE_TRY(step_real_dev(p, p->host_buf, nsteps));
    GPE_CUDA(cudaMemcpyAsync(psi_host, p->host_buf, bytes, cudaMemcpyDeviceToHost, p->st));
    return check_err(p);
}

// ------------------------------------------------------------------ diagnostics
// norm/energy/rms of psi into p->out6 / p->out4 (device), enqueued on p->st;
// kinetic = false (rms sizes only) skips the transforms that the kinetic
// energy needs (out6 then holds no valid energies)
static gpe_status diag_dev(gpe_plan *p, const void *psi, bool kinetic = true)
{
    const int64_t B = active_count(p);
    PassArgs x = make_pass(p, 0, psi, nullptr, B);
    x.red = kinetic ? RED_DIAG_X : RED_DIAG_XM;
    GPE_TRY(run(p, x));
    for (int a = 1; a < p->ndim && kinetic; ++a) {
        PassArgs k = make_pass(p, a, psi, nullptr, B);
        k.red = RED_DIAG_K;
        GPE_TRY(run(p, k));
    }
    const int *stop = p->cur_stop;
    cudaError_t e = launch_reduce_lines(p->partials, p->lines_cap, 0, 7, B, p->N / p->n[0], p->csum, p->sums, p->st,
                                        0.0, 0.0, nullptr, nullptr, stop);
    for (int a = 1; a < p->ndim && e == cudaSuccess && kinetic; ++a)
        e = launch_reduce_lines(p->partials, p->lines_cap, 6 + a, 1, B, p->N / p->n[a], p->csum, p->sums, p->st,
                                0.0, 0.0, nullptr, nullptr, stop);
    if (e == cudaSuccess)
        e = launch_finish_diag(p->sums, B, p->ndim, p->n, p->dv, p->g_dev, p->out6, p->out4, p->st, stop);
    if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("diagnostics: ") + cudaGetErrorString(e));
    return GPE_OK;
}

// copy results out; the stream is synchronised and the device error word checked
static gpe_status copy_out(gpe_plan *p, const double *dev, size_t count, double *host)
{
    GPE_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, p->st));
    return check_err(p);
}

extern "C" gpe_status gpe_plan_set_option(gpe_plan *p, int option, int64_t value)
{
    if (!p) return fail(GPE_EINVAL, "NULL plan");
    if (value != 0 && value != 1) return fail(GPE_EINVAL, "plan options take 0 or 1");
    if (option == GPE_OPT_TEST_STALL_COPIES) {
        p->tx_extra = value ? 16 : 0;
        return GPE_OK;
    }
    if (option == GPE_OPT_TMA_STAGING) {
        for (int a = 0; a < 3; ++a) p->use_tma[a] = value != 0;
        return GPE_OK;
    }
    if (option >= GPE_OPT_TILE_X && option <= GPE_OPT_TILE_Z) {
        p->tile_var[option - GPE_OPT_TILE_X] = (int)value;
        return GPE_OK;
    }
    if (option == GPE_OPT_TMA_Y || option == GPE_OPT_TMA_Z) {
        p->use_tma[option - GPE_OPT_TMA_Y + 1] = value != 0;
        return GPE_OK;
    }
    if (option == GPE_OPT_GENERIC_PASSES) {
        p->generic_passes = value != 0;
        return GPE_OK;
    }
    if (option == GPE_OPT_NO_DITHER) {
        p->no_dither = value != 0;
        return GPE_OK;
    }
    if (option == GPE_OPT_LINE_CLUSTER) {
        p->line_cluster = value != 0;
        return GPE_OK;
    }
    return fail(GPE_EINVAL, "unknown plan option");
}

extern "C" gpe_status gpe_plan_get_option(const gpe_plan *p, int option, int64_t *value)
{
    if (!p || !value) return fail(GPE_EINVAL, "NULL argument");
    if (option == GPE_OPT_TMA_STAGING) *value = (p->use_tma[1] || p->use_tma[2]) ? 1 : 0;
    else if (option >= GPE_OPT_TILE_X && option <= GPE_OPT_TILE_Z) *value = p->tile_var[option - GPE_OPT_TILE_X];
    else if (option == GPE_OPT_TMA_Y || option == GPE_OPT_TMA_Z) *value = p->use_tma[option - GPE_OPT_TMA_Y + 1] ? 1 : 0;
    else if (option == GPE_OPT_TEST_STALL_COPIES) *value = p->tx_extra ? 1 : 0;
    else if (option == GPE_OPT_GENERIC_PASSES) *value = p->generic_passes ? 1 : 0;
    else if (option == GPE_OPT_NO_DITHER) *value = p->no_dither ? 1 : 0;
    else if (option == GPE_OPT_LINE_CLUSTER) *value = p->line_cluster ? 1 : 0;
    else return fail(GPE_EINVAL, "unknown plan option");
    return GPE_OK;
}

// ------------------------------------------------------------------ autotuner
namespace {
struct TuneVal {
    int var[3];
    bool tma[3];
};
std::mutex g_tune_mu;
std::map<std::string, TuneVal> g_tune;   // choices per grid/precision/instances/flags, process-wide
}  // namespace

static std::string tune_key(const gpe_plan *p, int64_t batch, int flags)
{
    char buf[160];
    snprintf(buf, sizeof(buf), "%d/%d/%lldx%lldx%lld/%lld/%d", p->prec, p->ndim, (long long)p->n[0],
             (long long)p->n[1], (long long)p->n[2], (long long)batch, flags);
    return buf;
}

// the pass that the steady real-time step makes along `axis`
static PassArgs steady_pass(const gpe_plan *p, int axis, void *buf, int64_t batch)
{
    PassArgs a = make_pass(p, axis, buf, buf, batch);
    const int piv = p->ndim - 1;
    if (axis == 0) {
        a.fft1 = +1;
        a.op_mid = OP_NREAL;
        set_nreal(p, a, true);
        a.fft2 = -1;
    } else if (axis == piv) {
        a.fft1 = -1;
        a.op_mid = OP_KREAL;
        a.fft2 = +1;
    } else {
        a.fft1 = +1;
    }
    return a;
}

static void apply_tune(gpe_plan *p, const TuneVal &v)
{
    for (int a = 0; a < 3; ++a) {
        p->tile_var[a] = v.var[a];
        p->use_tma[a] = v.tma[a];
    }
}

extern "C" gpe_status gpe_plan_autotune(gpe_plan *p, const void *psi, int reps, int flags)
{
    if (!p) return fail(GPE_EINVAL, "NULL plan");
    if (psi && ((uintptr_t)psi) % 16 != 0) return fail(GPE_EINVAL, "psi must be 16-byte aligned");
    if (reps < 1 || reps > 1000) return fail(GPE_EINVAL, "reps must be in [1, 1000]");
    if (flags & ~GPE_TUNE_NO_TMA) return fail(GPE_EINVAL, "unknown autotune flag");
    if (p->ndim == 1) return GPE_OK;
    if (p->cur_count > 0) return fail(GPE_EINVAL, "plan is in use by a batch launch");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(GPE_ECUDA, "cannot select the plan's device");
    const int64_t B = p->batch;
    const std::string key = tune_key(p, B, flags);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply_tune(p, it->second);
            return GPE_OK;
        }
    }
    // Candidates are timed as whole steady steps on the state a step meets:
    // prep holds psi advanced through a real-time call's prologue, and buf
    // gets a fresh copy of prep before every timed step.  (The x pass in
    // particular must see physical |psi|: its nonlinear phase takes a cheaper
    // path for small angles.)
    const size_t bytes = (size_t)B * (size_t)p->N * p->csize;
    void *buf = nullptr, *prep = nullptr;
    GPE_CUDA(cudaMalloc(&buf, bytes));
    if (cudaMalloc(&prep, bytes) != cudaSuccess) {
        cudaFree(buf);
        return fail(GPE_ENOMEM, "autotune scratch");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gpe_status st = GPE_OK;
    TuneVal best;
    for (int a = 0; a < 3; ++a) {
        best.var[a] = 0;
        best.tma[a] = a >= 1 && !(flags & GPE_TUNE_NO_TMA);
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = fail(GPE_ECUDA, "cudaEventCreate failed");
    if (st == GPE_OK) {
        cudaError_t e = psi ? cudaMemcpyAsync(prep, psi, bytes, cudaMemcpyDeviceToDevice, p->st)
                            : cudaMemsetAsync(prep, 0, bytes, p->st);
        if (e != cudaSuccess) st = fail(GPE_ECUDA, "scratch set-up failed");
    }
    // prologue of a real-time step: first nonlinear half-step with FFT_x, then FFT_y (3D)
    if (st == GPE_OK) {
        PassArgs x0 = make_pass(p, 0, prep, prep, B);
        x0.op_pre = OP_NREAL;
        set_nreal(p, x0, false);
        x0.fft1 = -1;
        st = run(p, x0);
    }
    if (st == GPE_OK && p->ndim == 3) {
        PassArgs y = make_pass(p, 1, prep, prep, B);
        y.fft1 = -1;
        st = run(p, y);
    }
    const int piv = p->ndim - 1;
    // one steady real-time step on b (state in mixed space, as prep is after
    // the prologue): the pivot pass (F K I), y inverse (3D), x (I N F), y forward (3D)
    auto run_step = [&](void *b) -> gpe_status {
        GPE_TRY(run(p, steady_pass(p, piv, b, B)));
        if (p->ndim == 3) GPE_TRY(run(p, steady_pass(p, 1, b, B)));
        GPE_TRY(run(p, steady_pass(p, 0, b, B)));
        if (p->ndim == 3) {
            PassArgs yf = make_pass(p, 1, b, b, B);
            yf.fft1 = -1;
            GPE_TRY(run(p, yf));
        }
        return GPE_OK;
    };
    // Axes in the step's order (3D: z, y, x; 2D: y, x).  Each candidate
    // (shape, staging) of an axis is timed as a whole step, with the other
    // axes at their current choice, from a fresh copy of prep; candidates
    // are taken round-robin and ranked by their fastest step.  Timing the
    // pass alone, after the copy, favoured the 16-line 512^3 z tile, which is
    // the slower one inside the step (0.784 against 0.759 ms: the overlap of
    // consecutive launches differs between the shapes); summed sequential
    // timings also let clock drift between candidates decide.
    // two sweeps over the axes: a shape's speed depends on its neighbours' (the
    // overlap of consecutive launches), so the axes tuned first are tuned again
    // with the others at their choice (the 512^3 z shape was picked against
    // the default y shape and lost 0.02 ms per step once y had its own)
    const int order[6] = {piv, 1, 0, piv, 1, 0};
    for (int a = 0; a < 3; ++a) {
        p->tile_var[a] = best.var[a];
        p->use_tma[a] = best.tma[a];
    }
    // steps per timed sample: about 2 ms of work, so that small grids are not
    // timed at the resolution of the events (one 1024^2 step is ~25 us)
    int k = 1;
    for (int r = 0; r < 2 && st == GPE_OK; ++r) {
        if (cudaMemcpyAsync(buf, prep, bytes, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess) {
            st = fail(GPE_ECUDA, "scratch copy failed");
            break;
        }
        cudaEventRecord(e0, p->st);
        st = run_step(buf);
        cudaEventRecord(e1, p->st);
        float ms = 0.f;
        if (st == GPE_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = fail(GPE_ECUDA, "timing a step failed");
        if (st == GPE_OK && r == 1) k = ms > 0.f ? (int)std::min(64.0, std::max(1.0, 2.0 / (double)ms)) : 64;
    }
    for (int oi = 0; oi < 6 && st == GPE_OK; ++oi) {
        const int a = order[oi];
        if (oi % 3 == 1 && p->ndim != 3) continue;     // 2D: the pivot is y, already tuned in this sweep
        const int ntma = (a >= 1 && !(flags & GPE_TUNE_NO_TMA)) ? 2 : 1;
        const int ncand = 2 * ntma;
        double cand_ms[4] = {1e300, 1e300, 1e300, 1e300};
        for (int r = 0; r <= reps && st == GPE_OK; ++r) {       // r = 0 warms every candidate up
            for (int c = 0; c < ncand && st == GPE_OK; ++c) {
                p->tile_var[a] = c / ntma;
                p->use_tma[a] = ntma == 2 && c % ntma == 0;
                if (cudaMemcpyAsync(buf, prep, bytes, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess) {
                    st = fail(GPE_ECUDA, "scratch copy failed");
                    break;
                }
                // one untimed step first: the copy leaves the end of the state in
                // L2, which the first pass after it would otherwise meet
                st = run_step(buf);
                if (st != GPE_OK) break;
                cudaEventRecord(e0, p->st);
                for (int i = 0; i < k && st == GPE_OK; ++i) st = run_step(buf);
                cudaEventRecord(e1, p->st);
                if (st != GPE_OK) break;
                float ms = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    st = fail(GPE_ECUDA, "timing the candidate failed");
                    break;
                }
                if (r > 0) cand_ms[c] = std::min(cand_ms[c], (double)ms);
            }
        }
        double best_ms = 1e300;
        for (int c = 0; c < ncand && st == GPE_OK; ++c) {
            if (cand_ms[c] < best_ms) {
                best_ms = cand_ms[c];
                best.var[a] = c / ntma;
                best.tma[a] = ntma == 2 && c % ntma == 0;
            }
        }
        p->tile_var[a] = best.var[a];
        p->use_tma[a] = best.tma[a];
    }
    cudaFree(prep);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (st == GPE_OK) st = check_err(p);
    if (st != GPE_OK) {
        TuneVal d;
        for (int a = 0; a < 3; ++a) {
            d.var[a] = 0;
            d.tma[a] = true;
        }
        apply_tune(p, d);
        return st;
    }
    apply_tune(p, best);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = best;
    return GPE_OK;
}

extern "C" gpe_status gpe_norm_energy(gpe_plan *p, const void *psi, double *out)
{
    GPE_TRY(check_psi(p, psi));
    if (!out) return fail(GPE_EINVAL, "NULL output");
    DeviceGuard dg(p->device);
    GPE_TRY(diag_dev(p, psi));
    return copy_out(p, p->out6, 6 * (size_t)p->batch, out);
}

extern "C" gpe_status gpe_rms_size(gpe_plan *p, const void *psi, double *out)
{
    GPE_TRY(check_psi(p, psi));
    if (!out) return fail(GPE_EINVAL, "NULL output");
    DeviceGuard dg(p->device);
    GPE_TRY(diag_dev(p, psi, false));
    return copy_out(p, p->out4, 4 * (size_t)p->batch, out);
}

// ------------------------------------------------------------------ imaginary time
// renormalisation factors back to one (a device-to-device copy: no host wait)
static gpe_status fill_scale_one(gpe_plan *p)
{
    GPE_CUDA(cudaMemcpyAsync(p->scale, p->ones, sizeof(double) * p->batch, cudaMemcpyDeviceToDevice, p->st));
    return GPE_OK;
}

static gpe_status imag_steps(gpe_plan *p, void *psi, int64_t nsteps, double target)
{
    const int64_t B = active_count(p);
    if (nsteps <= 0) return GPE_OK;
    if (p->ndim == 1) {
        Line1DArgs l;
        memset(&l, 0, sizeof(l));
        l.psi = psi;
        l.batch = B;
        l.n = (int)p->n[0];
        l.nsteps = nsteps;
        l.imag = 1;
        l.tw = p->tw[0];
        l.kt = p->ki[0];
        l.vi = p->vi[0];
        l.g = p->g_dev;
        l.dt = p->dt;
        l.target_norm_over_dv = target / p->dv;
        l.err = p->err;
        l.stop = p->cur_stop;
        if (p->cur_count > 0) {
            l.inst_ptr = p->cur_ptrs;
            l.slot_of = p->cur_slots;
        }
        TraceScope ts(p, "line1d" + std::to_string(l.n) + ":imag");
        cudaError_t e = launch_line1d(p->prec, l, p->st);
        if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("1D launch: ") + cudaGetErrorString(e));
        return GPE_OK;
    }
    GPE_TRY(fill_scale_one(p));
    const int piv = p->ndim - 1;
    for (int64_t s = 0; s < nsteps; ++s) {
        PassArgs x = make_pass(p, 0, psi, psi, B);
        x.op_pre = OP_SCALE_NIMAG;
        x.nl_c = 0.5 * p->dt;
        x.fft1 = -1;
        GPE_TRY(run(p, x));
        if (p->ndim == 3) {
            PassArgs y = make_pass(p, 1, psi, psi, B);
            y.fft1 = -1;
            GPE_TRY(run(p, y));
        }
        PassArgs k = make_pass(p, piv, psi, psi, B);
        k.fft1 = -1;
        k.op_mid = OP_KIMAG;
        k.fft2 = +1;
        GPE_TRY(run(p, k));
        if (p->ndim == 3) {
            PassArgs y = make_pass(p, 1, psi, psi, B);
            y.fft1 = +1;
            GPE_TRY(run(p, y));
        }
        PassArgs x2 = make_pass(p, 0, psi, psi, B);
        x2.fft1 = +1;
        x2.op_mid = OP_NIMAG;
        x2.nl_c = 0.5 * p->dt;
        x2.red = RED_NORM;
        GPE_TRY(run(p, x2));
        cudaError_t e = launch_reduce_lines(p->partials, p->lines_cap, 0, 1, B, p->N / p->n[0], p->csum, p->sums,
                                            p->st, p->dv, target, p->scale, p->err, p->cur_stop);
        if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("renormalisation: ") + cudaGetErrorString(e));
    }
    // apply the last renormalisation
    PassArgs xs = make_pass(p, 0, psi, psi, B);
    xs.op_pre = OP_SCALE;
    GPE_TRY(run(p, xs));
    return GPE_OK;
}

static gpe_status check_err(gpe_plan *p)
{
    int h = 0;
    GPE_CUDA(cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    GPE_CUDA(cudaStreamSynchronize(p->st));
    if (h) {
        cudaMemsetAsync(p->err, 0, sizeof(int), p->st);
        cudaStreamSynchronize(p->st);
        if (h & ERR_TMA_TIMEOUT) return fail(GPE_ETIMEOUT, "a tile copy did not complete within the wait limit");
        if (h & ERR_CLUSTER_TIMEOUT)
            return fail(GPE_ETIMEOUT, "an exchange between the CTAs of a cluster did not complete within the wait limit");
        return fail(GPE_ENUMERIC, "norm became zero or non-finite during imaginary time");
    }
    return GPE_OK;
}

extern "C" gpe_status gpe_step_imag(gpe_plan *p, void *psi, int64_t max_steps, double target_norm, double etol,
                                    int check_every, int64_t *steps_done, double *E_final)
{
    GPE_TRY(check_psi(p, psi));
    if (max_steps < 0) return fail(GPE_EINVAL, "max_steps must be >= 0");
    if (check_every < 1) return fail(GPE_EINVAL, "check_every must be >= 1");
    if (!(target_norm > 0.0) || !isfinite(target_norm)) return fail(GPE_EINVAL, "target_norm must be positive");
    DeviceGuard dg(p->device);
    const int64_t B = p->batch;
    int *d_stop = reinterpret_cast<int *>(p->istate);
    int64_t *d_done = reinterpret_cast<int64_t *>(p->istate + 8);
    // first reference energies, stop word and step counter on the device
    GPE_TRY(diag_dev(p, psi));
    cudaError_t e = launch_imag_init(p->out6, p->eprev, B, d_stop, d_done, p->st);
    if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("imaginary time: ") + cudaGetErrorString(e));
    // Chunks of check_every steps, each followed by the diagnostics and the
    // device-side test, are enqueued a window at a time without waiting; the
    // host reads the stop word and step counter once per window.  Once the
    // test has fired, the kernels of the chunks still queued see the stop
    // word and do nothing, so the state, step count and energy are those of
    // the check that stopped the run: the rule of a host-side loop.
    struct StopGuard {
        gpe_plan *p;
        ~StopGuard() { p->cur_stop = nullptr; }
    } guard{p};
    p->cur_stop = d_stop;
    unsigned char *hp = reinterpret_cast<unsigned char *>(p->pin + 6 * B);
    int64_t queued = 0, window = 2;
    int h_stop = 0;
    int64_t h_done = 0;
    while (true) {
        for (int64_t w = 0; w < window && queued < max_steps; ++w) {
            const int64_t chunk = std::min<int64_t>(check_every, max_steps - queued);
            GPE_TRY(imag_steps(p, psi, chunk, target_norm));
            GPE_TRY(diag_dev(p, psi));
            e = launch_imag_check(p->out6, p->eprev, B, etol, chunk, d_stop, d_done, p->err, p->st);
            if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("imaginary time: ") + cudaGetErrorString(e));
            queued += chunk;
        }
        GPE_CUDA(cudaMemcpyAsync(hp, p->istate, 16, cudaMemcpyDeviceToHost, p->st));
        GPE_TRY(check_err(p));     // synchronises
        memcpy(&h_stop, hp, sizeof(int));
        memcpy(&h_done, hp + 8, sizeof(int64_t));
        if (h_stop == 2) return fail(GPE_ENUMERIC, "energy or norm became non-finite or zero during imaginary time");
        if (h_stop == 1 || queued >= max_steps) break;
        window = std::min<int64_t>(2 * window, 16);   // longer runs: fewer round trips
    }
    p->cur_stop = nullptr;
    if (steps_done) *steps_done = h_done;
    if (E_final) {
        GPE_CUDA(cudaMemcpyAsync(p->pin, p->eprev, sizeof(double) * B, cudaMemcpyDeviceToHost, p->st));
        GPE_CUDA(cudaStreamSynchronize(p->st));
        for (int64_t b = 0; b < B; ++b) E_final[b] = p->pin[b];
    }
    return GPE_OK;
}

// ------------------------------------------------------------------ spectra
static int64_t nshells_of(const gpe_plan *p)
{
    double lmax = 0.0;
    for (int a = 0; a < p->ndim; ++a) lmax = std::max(lmax, p->len[a]);
    double q2 = 0.0;
    for (int a = 0; a < p->ndim; ++a) {
        const double q = (double)(p->n[a] / 2) * (lmax / p->len[a]);
        q2 += q * q;
    }
    return (int64_t)floor(sqrt(q2) + 0.5) + 1;
}

extern "C" int64_t gpe_spectrum_nshells(const gpe_plan *p)
{
    if (!p) return -1;
    return nshells_of(p);
}

// forward (dir=-1) or inverse (+1) transform of one instance over all axes, src -> dst
static gpe_status fft_nd(gpe_plan *p, const void *src, void *dst, int dir)
{
    for (int a = 0; a < p->ndim; ++a) {
        PassArgs t = make_pass(p, a, a == 0 ? src : dst, dst, 1);
        t.fft1 = dir;
        GPE_TRY(run(p, t));
    }
    return GPE_OK;
}

extern "C" gpe_status gpe_spectrum(gpe_plan *p, const void *psi, unsigned kinds, double *out, int64_t nshells)
{
    GPE_TRY(check_psi(p, psi));
    if (!out) return fail(GPE_EINVAL, "NULL output");
    const unsigned all = GPE_SPEC_INC | GPE_SPEC_COMP | GPE_SPEC_QP | GPE_SPEC_NUM;
    if (!(kinds & all) || (kinds & ~all))
        return fail(GPE_EINVAL, "kinds must be a non-empty combination of GPE_SPEC_INC, GPE_SPEC_COMP, "
                                "GPE_SPEC_QP and GPE_SPEC_NUM");
    const int64_t ns = nshells_of(p);
    if (nshells < ns) return fail(GPE_EINVAL, "nshells smaller than gpe_spectrum_nshells()");
    if (ns > 6144) return fail(GPE_EUNSUPPORTED, "too many spectral shells");
    DeviceGuard dg(p->device);
    SpecArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.prec = p->prec;
    sa.ndim = p->ndim;
    double lmax = 0.0;
    for (int a = 0; a < p->ndim; ++a) lmax = std::max(lmax, p->len[a]);
    for (int a = 0; a < 3; ++a) {
        sa.n[a] = p->n[a];
        sa.kf[a] = p->kf[a];
        sa.lratio[a] = a < p->ndim ? lmax / p->len[a] : 0.0;
    }
    sa.N = p->N;
    const size_t field = (size_t)p->N * p->csize;
    if (!p->work[0]) {
        for (int w = 0; w <= p->ndim; ++w) GPE_TRY(dalloc(p, &p->work[w], field));
    }
    const int nb = bin_blocks(sa);
    if (!p->hist || p->nshells < ns || p->hist_blocks < nb) {
        // block histograms, then the fixed-point total partials and scale
        GPE_TRY(dalloc(p, (void **)&p->hist, sizeof(double) * (2 * (size_t)ns * nb + nb + 1)));
        GPE_TRY(dalloc(p, (void **)&p->spec_out, sizeof(double) * 2 * (size_t)ns));
        p->nshells = ns;
        p->hist_blocks = nb;
    }
    // output slot of each kind: requested kinds in bit order
    double *slot[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<double> tmp(2 * ns);
    // bin the given fields and write shells (scaled) into o0 / o1 (either may be NULL)
    auto bin_out = [&](void *const *uh, int split, int ncomp, double scale, double *o0, double *o1) -> gpe_status {
        SpecArgs sb = sa;
        sb.split = split;
        sb.ncomp = ncomp;
        double *aux = p->hist + 2 * (size_t)ns * nb;
        cudaError_t e = launch_bin(sb, uh, ns, p->hist, nb, aux, p->st);
        if (e == cudaSuccess)
            e = launch_hist_reduce(p->hist, nb, ns, p->dv / (double)p->N, aux, p->spec_out, p->spec_out + ns,
                                   p->st);
        if (e != cudaSuccess) return fail(GPE_ECUDA, cudaGetErrorString(e));
        GPE_CUDA(cudaMemcpyAsync(tmp.data(), p->spec_out, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, p->st));
        GPE_CUDA(cudaStreamSynchronize(p->st));
        double *o[2] = {o0, o1};
        for (int k = 0; k < 2; ++k)
            if (o[k])
                for (int64_t s2 = 0; s2 < nshells; ++s2) o[k][s2] = s2 < ns ? scale * tmp[k * ns + s2] : 0.0;
        return GPE_OK;
    };
    // derivative fields -> u (part 0) or w (part 1) -> their transforms, in work[1..ndim]
    auto gradient_parts = [&](const void *pb, int part) -> gpe_status {
        SpecArgs sv = sa;
        sv.part = part;
        for (int a = 0; a < p->ndim; ++a) {
            cudaError_t e = launch_deriv(sa, p->work[0], p->work[1 + a], a, p->st);
            if (e != cudaSuccess) return fail(GPE_ECUDA, cudaGetErrorString(e));
            GPE_TRY(fft_nd(p, p->work[1 + a], p->work[1 + a], +1));
            e = launch_velocity(sv, pb, p->work[1 + a], p->st);
            if (e != cudaSuccess) return fail(GPE_ECUDA, cudaGetErrorString(e));
            GPE_TRY(fft_nd(p, p->work[1 + a], p->work[1 + a], -1));
        }
        return GPE_OK;
    };
    void *uh[3] = {p->work[1], p->ndim > 1 ? p->work[2] : nullptr, p->ndim > 2 ? p->work[3] : nullptr};
    for (int64_t b = 0; b < p->batch; ++b) {
        int kslot = 0;
        for (int k = 0; k < 4; ++k) {
            slot[k] = nullptr;
            if (kinds & (1u << k)) slot[k] = out + ((size_t)kslot++ * p->batch + b) * nshells;
        }
        const char *pb = (const char *)psi + (size_t)b * field;
        GPE_TRY(fft_nd(p, pb, p->work[0], -1));
        if (slot[3]) {
            // the bins carry 1/2 dV/N; the number spectrum has no 1/2
            void *ph[3] = {p->work[0], nullptr, nullptr};
            GPE_TRY(bin_out(ph, 0, 1, 2.0, slot[3], nullptr));
        }
        if (slot[0] || slot[1]) {
            GPE_TRY(gradient_parts(pb, 0));
            GPE_TRY(bin_out(uh, 1, p->ndim, 1.0, slot[0], slot[1]));
        }
        if (slot[2]) {
            GPE_TRY(gradient_parts(pb, 1));
            GPE_TRY(bin_out(uh, 0, p->ndim, 1.0, slot[2], nullptr));
        }
    }
    return GPE_OK;
}

// ------------------------------------------------------------------ internal (serve.cu)
namespace gpe {

cudaStream_t plan_stream(const gpe_plan *p) { return p->st; }
int64_t plan_capacity(const gpe_plan *p) { return p->batch; }
int64_t plan_points(const gpe_plan *p) { return p->N; }
size_t plan_point_bytes(const gpe_plan *p) { return p->csize; }

// Resolve every kernel the plan will launch (function attributes, occupancy)
// with zero-work launches, so that later launches can be captured in graphs.
gpe_status plan_prepare(gpe_plan *p)
{
    DeviceGuard dg(p->device);
    for (int a = 0; a < p->ndim; ++a) {
        PassArgs t = make_pass(p, a, nullptr, nullptr, 0);
        t.ntiles = 0;
        cudaError_t e = launch_pass(p->prec, a == 0, t, p->st);
        if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("prepare: ") + cudaGetErrorString(e));
    }
    if (p->ndim == 1) {
        Line1DArgs l;
        memset(&l, 0, sizeof(l));
        l.n = (int)p->n[0];
        l.batch = 0;
        cudaError_t e = launch_line1d(p->prec, l, p->st);
        if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("prepare: ") + cudaGetErrorString(e));
    }
    return GPE_OK;
}

// Give slot `slot` of a plan new interaction and trap parameters: host FP64
// tables, uploaded on the plan stream.  Axes without a trap table keep none
// (the caller groups instances by which axes are trapped).
gpe_status plan_set_slot(gpe_plan *p, int64_t slot, double g, const double *gamma)
{
    if (slot < 0 || slot >= p->batch) return fail(GPE_EINVAL, "slot out of range");
    DeviceGuard dg(p->device);
    GPE_CUDA(cudaMemcpyAsync(p->g_dev + slot, &g, sizeof(double), cudaMemcpyHostToDevice, p->st));
    double gm[3] = {0, 0, 0};
    for (int a = 0; a < p->ndim; ++a) gm[a] = gamma[a];
    GPE_CUDA(cudaMemcpyAsync(p->gamma_dev + 3 * slot, gm, sizeof(gm), cudaMemcpyHostToDevice, p->st));
    for (int a = 0; a < p->ndim; ++a) {
        if (!p->trap[a]) continue;
        const int64_t na = p->n[a];
        std::vector<double> vh(2 * na), vf(2 * na), vi(na);
        trap_tables_host(p, a, gm[a], vh.data(), vf.data(), vi.data());
        std::vector<unsigned char> bh, bf;
        pack_cplx(p, vh, bh);
        pack_cplx(p, vf, bf);
        const size_t ce = bh.size() / (size_t)na;      // bytes per complex entry
        GPE_CUDA(cudaMemcpyAsync((char *)p->vh[a] + slot * na * ce, bh.data(), bh.size(), cudaMemcpyHostToDevice, p->st));
        GPE_CUDA(cudaMemcpyAsync((char *)p->vf[a] + slot * na * ce, bf.data(), bf.size(), cudaMemcpyHostToDevice, p->st));
        if (p->prec == GPE_C64) {
            std::vector<float> f(vi.begin(), vi.end());
            GPE_CUDA(cudaMemcpyAsync((float *)p->vi[a] + slot * na, f.data(), f.size() * sizeof(float),
                                     cudaMemcpyHostToDevice, p->st));
            GPE_CUDA(cudaStreamSynchronize(p->st));    // host staging goes out of scope
        } else {
            GPE_CUDA(cudaMemcpyAsync((double *)p->vi[a] + slot * na, vi.data(), vi.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, p->st));
            GPE_CUDA(cudaStreamSynchronize(p->st));
        }
    }
    GPE_CUDA(cudaStreamSynchronize(p->st));
    return GPE_OK;
}

// Run `count` instances found through the device arrays dptrs (base pointers)
// and dslots (parameter slots): mode 0 = nsteps real-time steps, 1 = nsteps
// imaginary-time steps renormalised to target, 2 = diagnostics into
// out6_host[6*count] (norm, E_kin, E_pot, E_int, E, mu).
gpe_status plan_run(gpe_plan *p, int mode, void *const *dptrs, const int *dslots, int64_t count, int64_t nsteps,
                    double target, double *out6_host)
{
    if (count < 1 || count > p->batch) return fail(GPE_EINVAL, "instance count out of range");
    DeviceGuard dg(p->device);
    p->cur_ptrs = dptrs;
    p->cur_slots = dslots;
    p->cur_count = count;
    gpe_status s = GPE_OK;
    void *psi = const_cast<void *>(static_cast<const void *>(dptrs));
    if (mode == 0) s = step_real_dev(p, psi, nsteps);
    else if (mode == 1) {
        s = imag_steps(p, psi, nsteps, target);
        if (s == GPE_OK) s = check_err(p);
    } else {
        s = diag_dev(p, psi);
        if (s == GPE_OK) s = copy_out(p, p->out6, 6 * (size_t)count, out6_host);
    }
    p->cur_ptrs = nullptr;
    p->cur_slots = nullptr;
    p->cur_count = 0;
    return s;
}

// Resident path for batches of small 2D complex64 instances: the dither
// table (the values step_real_dev passes to its launches) once per plan, then
// one launch that runs every step of the call on chip.
bool plan_resident_ok(const gpe_plan *p) { return resident2d_supported(p->prec == GPE_C64 ? 0 : 1, p->ndim, p->n) && !p->vsamp; }

gpe_status plan_prepare_resident(gpe_plan *p)
{
    if (p->dtab) return GPE_OK;
    DeviceGuard dg(p->device);
    std::vector<double> h(5 * (size_t)GPE_DITHER_PERIOD);
    for (int64_t s = 0; s < GPE_DITHER_PERIOD; ++s) {
        PassArgs k;
        memset(&k, 0, sizeof(k));
        const double phi = dither_angle(s);
        set_dither(k, phi);
        h[5 * s] = phi;
        for (int q = 0; q < 4; ++q) h[5 * s + 1 + q] = k.dk[q];
    }
    GPE_TRY(dalloc(p, (void **)&p->dtab, sizeof(double) * h.size()));
    GPE_CUDA(cudaMemcpy(p->dtab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
    return GPE_OK;
}

gpe_status plan_run_resident(gpe_plan *p, void *const *dptrs, const int *dslots, int64_t count, int64_t nsteps)
{
    if (!plan_resident_ok(p) || !p->dtab) return fail(GPE_EUNSUPPORTED, "resident path not prepared for this plan");
    if (count < 1 || count > p->batch) return fail(GPE_EINVAL, "instance count out of range");
    if (nsteps <= 0) return GPE_OK;
    DeviceGuard dg(p->device);
    ResidentArgs r;
    memset(&r, 0, sizeof(r));
    r.inst_ptr = dptrs;
    r.slot_of = dslots;
    r.count = count;
    r.nsteps = nsteps;
    r.tw = p->tw[0];
    r.rows = make_pass(p, 0, nullptr, nullptr, count);
    set_nreal(p, r.rows, true);
    r.rows.op_mid = OP_NREAL;
    r.cols = make_pass(p, 1, nullptr, nullptr, count);
    r.cols.op_mid = OP_KREAL;
    for (int a = 0; a < 2; ++a) {
        r.vh[a] = p->vh[a];
        r.vf[a] = p->vf[a];
    }
    r.dt = p->dt;
    r.dither = p->prec == GPE_C64 && !p->no_dither;
    r.dtab = p->dtab;
    TraceScope ts(p, "resident2d" + std::to_string(p->n[0]) + ":real");
    cudaError_t e = launch_resident2d((int)p->n[0], r, p->st);
    if (e != cudaSuccess) return fail(GPE_ECUDA, std::string("resident launch: ") + cudaGetErrorString(e));
    return GPE_OK;
}

// The same without waiting: mode 1 enqueues nsteps imaginary-time steps and
// then the diagnostics, mode 2 only the diagnostics; out6 (6*count doubles)
// and the device error word are copied into the pinned host buffers out6_pin
// and err_pin, and the error word is cleared.  The caller synchronises the
// plan stream before it reads them.
gpe_status plan_run_async(gpe_plan *p, int mode, void *const *dptrs, const int *dslots, int64_t count, int64_t nsteps,
                          double target, double *out6_pin, int *err_pin)
{
    if (count < 1 || count > p->batch) return fail(GPE_EINVAL, "instance count out of range");
    DeviceGuard dg(p->device);
    p->cur_ptrs = dptrs;
    p->cur_slots = dslots;
    p->cur_count = count;
    gpe_status s = GPE_OK;
    void *psi = const_cast<void *>(static_cast<const void *>(dptrs));
    if (mode == 1) s = imag_steps(p, psi, nsteps, target);
    if (s == GPE_OK) s = diag_dev(p, psi);
    if (s == GPE_OK &&
        (cudaMemcpyAsync(out6_pin, p->out6, sizeof(double) * 6 * count, cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
         cudaMemcpyAsync(err_pin, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
         cudaMemsetAsync(p->err, 0, sizeof(int), p->st) != cudaSuccess))
        s = fail(GPE_ECUDA, "copying results back failed");
    p->cur_ptrs = nullptr;
    p->cur_slots = nullptr;
    p->cur_count = 0;
    return s;
}

}  // namespace gpe
