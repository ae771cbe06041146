// serve.cu - batches of independent GPE instances and a continuous-batching
// request server, on top of the plan drivers in api.cu.
//
// Instances that share grid, box, time step, precision and trapped axes share
// one plan ("group"): their states are separate device buffers, reached
// through a device array of base pointers, and their interaction and trap
// parameters sit in per-slot tables, so every pass of a step covers all of a
// group's instances in one launch.  Different groups run on their own
// streams, forked from and joined back to the caller's stream.
//
// Splitting a run into chunks of whole steps is exact (each chunk starts and
// ends with a nonlinear half-step, and consecutive halves compose to the full
// step), so the server can let requests join and leave between chunks.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gpe.h"
#include "../../include/gpe_serve.h"
#include "gpe_internal.h"

namespace gpe {
cudaStream_t plan_stream(const gpe_plan *p);
int64_t plan_capacity(const gpe_plan *p);
int64_t plan_points(const gpe_plan *p);
size_t plan_point_bytes(const gpe_plan *p);
gpe_status plan_set_slot(gpe_plan *p, int64_t slot, double g, const double *gamma);
gpe_status plan_prepare(gpe_plan *p);
gpe_status plan_run(gpe_plan *p, int mode, void *const *dptrs, const int *dslots, int64_t count, int64_t nsteps,
                    double target, double *out6_host);
gpe_status plan_run_async(gpe_plan *p, int mode, void *const *dptrs, const int *dslots, int64_t count, int64_t nsteps,
                          double target, double *out6_pin, int *err_pin);
bool plan_resident_ok(const gpe_plan *p);
gpe_status plan_prepare_resident(gpe_plan *p);
gpe_status plan_run_resident(gpe_plan *p, void *const *dptrs, const int *dslots, int64_t count, int64_t nsteps);
}  // namespace gpe

using namespace gpe;

namespace {

gpe_status sfail(gpe_status s, const std::string &msg)
{
    set_last_error(msg.c_str());
    return s;
}

#define S_CUDA(call)                                                                            \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return sfail(GPE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Instances with equal keys can share a plan.
std::string group_key(const gpe_plan_desc &d, int extra)
{
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append(static_cast<const char *>(p), n); };
    put(&d.ndim, sizeof(d.ndim));
    put(&d.prec, sizeof(d.prec));
    put(&extra, sizeof(extra));
    for (int a = 0; a < d.ndim; ++a) {
        put(&d.n[a], sizeof(d.n[a]));
        put(&d.lo[a], sizeof(double));
        put(&d.len[a], sizeof(double));
        const char trapped = d.gamma[a] != 0.0;
        put(&trapped, 1);
    }
    put(&d.dt, sizeof(double));
    return k;
}

gpe_status check_desc(const gpe_plan_desc &d)
{
    if (d.batch != 1) return sfail(GPE_EINVAL, "each instance description must have batch == 1");
    if (d.g_each || d.gamma_each) return sfail(GPE_EINVAL, "per-instance arrays are not used here");
    if (d.V_host) return sfail(GPE_EUNSUPPORTED, "sampled potentials are taken by single plans only");
    return GPE_OK;
}

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// ====================================================================== batch
struct BGroup {
    gpe_plan *plan = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool resident = false;         // small 2D complex64 instances: stepped on chip (resident.cu)
    std::vector<int> members;      // instance indices of the batch
    void **d_ptrs = nullptr;
    int *d_slots = nullptr;
};

struct gpe_batch {
    int device = 0;
    cudaStream_t st = nullptr;       // caller's stream
    cudaStream_t cap = nullptr;      // private stream that graphs are captured on
    cudaEvent_t fork = nullptr;
    int count = 0;
    std::vector<BGroup> groups;
    std::vector<void *> last_ptrs;
    std::map<int64_t, cudaGraphExec_t> graphs;
};

static void batch_free(gpe_batch *b)
{
    if (!b) return;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &g : b->groups) {
        if (g.plan) gpe_plan_destroy(g.plan);
        if (g.st) cudaStreamDestroy(g.st);
        if (g.done) cudaEventDestroy(g.done);
        if (g.d_ptrs) cudaFree(g.d_ptrs);
        if (g.d_slots) cudaFree(g.d_slots);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

extern "C" gpe_status gpe_batch_create(const gpe_plan_desc *descs, int count, void *cuda_stream, gpe_batch **out)
{
    if (!descs || !out || count < 1) return sfail(GPE_EINVAL, "gpe_batch_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        gpe_status s = check_desc(descs[i]);
        if (s != GPE_OK) return s;
    }
    gpe_batch *b = new gpe_batch();
    b->count = count;
    b->st = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&b->device) != cudaSuccess || cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b);
        return sfail(GPE_ECUDA, "gpe_batch_create: CUDA setup failed");
    }
    std::map<std::string, int> gi;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < count; ++i) {
        const std::string k = group_key(descs[i], 0);
        auto it = gi.find(k);
        if (it == gi.end()) {
            gi[k] = (int)members.size();
            members.push_back({i});
        } else {
            members[it->second].push_back(i);
        }
    }
    for (auto &m : members) {
        BGroup g;
        g.members = m;
        const int n = (int)m.size();
        gpe_plan_desc d = descs[m[0]];
        std::vector<double> ge(n), gm(3 * n);
        for (int j = 0; j < n; ++j) {
            ge[j] = descs[m[j]].g;
            for (int a = 0; a < 3; ++a) gm[3 * j + a] = a < d.ndim ? descs[m[j]].gamma[a] : 0.0;
        }
        d.batch = n;
        d.g_each = ge.data();
        d.gamma_each = gm.data();
        gpe_status s = GPE_OK;
        if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
            s = sfail(GPE_ECUDA, "stream creation failed");
        if (s == GPE_OK) s = gpe_plan_create(&d, g.st, &g.plan);
        // tile shapes timed on this group's grid (per-thread staging: the group's
        // instances are reached through a pointer array)
        if (s == GPE_OK) {
            g.resident = plan_resident_ok(g.plan);
            if (g.resident) s = plan_prepare_resident(g.plan);
            else s = gpe_plan_autotune(g.plan, nullptr, 3, GPE_TUNE_NO_TMA);
        }
        if (s == GPE_OK) s = plan_prepare(g.plan);
        if (s == GPE_OK && (cudaMalloc((void **)&g.d_ptrs, sizeof(void *) * n) != cudaSuccess ||
                            cudaMalloc((void **)&g.d_slots, sizeof(int) * n) != cudaSuccess))
            s = sfail(GPE_ENOMEM, "batch pointer arrays");
        if (s == GPE_OK) {
            std::vector<int> slots(n);
            for (int j = 0; j < n; ++j) slots[j] = j;
            if (cudaMemcpy(g.d_slots, slots.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess)
                s = sfail(GPE_ECUDA, "uploading slots failed");
        }
        b->groups.push_back(g);
        if (s != GPE_OK) {
            batch_free(b);
            return s;
        }
    }
    *out = b;
    return GPE_OK;
}

extern "C" gpe_status gpe_batch_destroy(gpe_batch *b)
{
    if (!b) return sfail(GPE_EINVAL, "NULL batch");
    cudaStreamSynchronize(b->st);
    batch_free(b);
    return GPE_OK;
}

static gpe_status batch_upload_ptrs(gpe_batch *b, void *const *psi)
{
    std::vector<void *> cur(psi, psi + b->count);
    if (cur == b->last_ptrs) return GPE_OK;
    for (int i = 0; i < b->count; ++i)
        if (!psi[i] || ((uintptr_t)psi[i]) % 16) return sfail(GPE_EINVAL, "instance pointers must be 16-byte aligned");
    S_CUDA(cudaStreamSynchronize(b->st));
    for (auto &g : b->groups) {
        std::vector<void *> h(g.members.size());
        for (size_t j = 0; j < h.size(); ++j) h[j] = psi[g.members[j]];
        S_CUDA(cudaMemcpy(g.d_ptrs, h.data(), sizeof(void *) * h.size(), cudaMemcpyHostToDevice));
    }
    b->last_ptrs = cur;
    return GPE_OK;
}

// fork the groups off `root`, run each group's nsteps, join back into `root`
static gpe_status batch_enqueue(gpe_batch *b, cudaStream_t root, int64_t nsteps)
{
    S_CUDA(cudaEventRecord(b->fork, root));
    for (auto &g : b->groups) {
        S_CUDA(cudaStreamWaitEvent(g.st, b->fork, 0));
        gpe_status s = g.resident
                           ? plan_run_resident(g.plan, g.d_ptrs, g.d_slots, (int64_t)g.members.size(), nsteps)
                           : plan_run(g.plan, 0, g.d_ptrs, g.d_slots, (int64_t)g.members.size(), nsteps, 1.0, nullptr);
        if (s != GPE_OK) return s;
        S_CUDA(cudaEventRecord(g.done, g.st));
        S_CUDA(cudaStreamWaitEvent(root, g.done, 0));
    }
    return GPE_OK;
}

extern "C" gpe_status gpe_batch_step_real(gpe_batch *b, void *const *psi_dev, int64_t nsteps, int use_graph)
{
    if (!b || !psi_dev) return sfail(GPE_EINVAL, "NULL argument");
    if (nsteps < 0) return sfail(GPE_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return GPE_OK;
    gpe_status s = batch_upload_ptrs(b, psi_dev);
    if (s != GPE_OK) return s;
    if (!use_graph) return batch_enqueue(b, b->st, nsteps);
    auto it = b->graphs.find(nsteps);
    if (it == b->graphs.end()) {
        cudaGraph_t graph = nullptr;
        S_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        s = batch_enqueue(b, b->cap, nsteps);
        cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (s != GPE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return sfail(GPE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return sfail(GPE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = b->graphs.emplace(nsteps, exec).first;
    }
    S_CUDA(cudaGraphLaunch(it->second, b->st));
    return GPE_OK;
}

extern "C" gpe_status gpe_batch_norm_energy(gpe_batch *b, void *const *psi_dev, double *out_host)
{
    if (!b || !psi_dev || !out_host) return sfail(GPE_EINVAL, "NULL argument");
    gpe_status s = batch_upload_ptrs(b, psi_dev);
    if (s != GPE_OK) return s;
    S_CUDA(cudaStreamSynchronize(b->st));
    for (auto &g : b->groups) {
        std::vector<double> o(6 * g.members.size());
        s = plan_run(g.plan, 2, g.d_ptrs, g.d_slots, (int64_t)g.members.size(), 0, 1.0, o.data());
        if (s != GPE_OK) return s;
        for (size_t j = 0; j < g.members.size(); ++j)
            memcpy(out_host + 6 * (size_t)g.members[j], &o[6 * j], 6 * sizeof(double));
    }
    return GPE_OK;
}

extern "C" int gpe_batch_groups(const gpe_batch *b) { return b ? (int)b->groups.size() : -1; }

// ====================================================================== server
namespace {

struct Req {
    uint64_t id = 0;
    gpe_request r{};
    std::vector<unsigned char> psi_host;   // initial state, then result
    std::string key;
    size_t bytes = 0;
    void *dpsi = nullptr;
    int slot = -1;
    int state = 0;                          // 0 queued, 1 active, 2 done
    int64_t done_steps = 0;
    double e_prev = 0.0;
    bool has_e0 = false;                    // imaginary time: energy of the input known
    gpe_result res{};
};

struct SGroup {
    gpe_plan *plan = nullptr;
    cudaStream_t st = nullptr;
    int imag = 0;
    std::vector<int> free_slots;
    std::vector<Req *> members;
    void **d_ptrs = nullptr;
    int *d_slots = nullptr;
    size_t bytes = 0;
    // pinned landing buffers of the energies and error words of one round's
    // launch sets (at most one set per member, plus the first-energy set)
    double *pin_out = nullptr;   // [6 * (2 cap + 1)]: every member at most twice per round
    int *pin_err = nullptr;      // [cap + 2]: one word per launch set
    int cap = 0;
};

}  // namespace

struct gpe_server {
    size_t budget = 0, used = 0;
    int max_active = 0, chunk = 64;
    int device = 0;
    cudaMemPool_t pool = nullptr;   // stream-ordered allocations of the request states
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::map<uint64_t, Req *> reqs;
    std::map<std::string, SGroup *> groups;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int active = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    gpe_status fatal = GPE_OK;
    std::string fatal_msg;
};

// device bytes of a group plan with `cap` slots (estimate used for admission)
static size_t group_bytes(const gpe_plan_desc &d, int cap)
{
    int64_t N = 1, nmin = 1 << 30, nsum = 0;
    for (int a = 0; a < d.ndim; ++a) {
        N *= d.n[a];
        nmin = std::min<int64_t>(nmin, d.n[a]);
        nsum += d.n[a];
    }
    const size_t lines = (size_t)(N / nmin) * cap;
    return lines * 9 * sizeof(double) + (size_t)cap * nsum * 64 + (size_t)nsum * 64 + 4096;
}

static gpe_status finish_req(gpe_server *s, SGroup *g, Req *r, gpe_status st)
{
    // result back to the host copy (its stream is idle here: the round has
    // synchronised it), device state returned to the pool without a device-wide wait
    if (r->dpsi) {
        cudaStream_t rs = g ? g->st : nullptr;
        if (st == GPE_OK && (cudaMemcpyAsync(r->psi_host.data(), r->dpsi, r->psi_host.size(), cudaMemcpyDeviceToHost,
                                             rs) != cudaSuccess ||
                             cudaStreamSynchronize(rs) != cudaSuccess))
            st = GPE_ECUDA;
        cudaFreeAsync(r->dpsi, rs);
        r->dpsi = nullptr;
    }
    if (g && r->slot >= 0) g->free_slots.push_back(r->slot);
    r->slot = -1;
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= r->bytes;
    s->active -= 1;
    r->res.status = st;
    r->res.steps_done = r->done_steps;
    r->res.t_done = now_s(s->t0);
    r->state = 2;
    s->cv_done.notify_all();
    return st;
}

// admit queued requests while slots and budget allow (worker thread)
static void admit(gpe_server *s)
{
    for (;;) {
        Req *r = nullptr;
        size_t extra = 0;
        SGroup *g = nullptr;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty() || s->active >= s->max_active) return;
            r = s->queue.front();
            auto it = s->groups.find(r->key);
            if (it != s->groups.end()) g = it->second;
            else extra = group_bytes(r->r.desc, s->max_active);
            if (s->used + r->bytes + extra > s->budget) {
                if (s->active > 0) return;              // wait for memory to free up
                s->queue.pop_front();
                r->res.status = GPE_EBUSY;
                r->res.t_done = now_s(s->t0);
                r->state = 2;
                s->cv_done.notify_all();
                continue;
            }
            s->queue.pop_front();
            s->used += r->bytes + extra;
            s->active += 1;
        }
        gpe_status st = GPE_OK;
        if (!g) {
            g = new SGroup();
            g->imag = r->r.imag;
            g->bytes = extra;
            gpe_plan_desc d = r->r.desc;
            d.batch = s->max_active;
            std::vector<double> ge(d.batch, d.g), gm(3 * (size_t)d.batch);
            for (int j = 0; j < d.batch; ++j)
                for (int a = 0; a < 3; ++a) gm[3 * j + a] = a < d.ndim ? d.gamma[a] : 0.0;
            d.g_each = ge.data();
            d.gamma_each = gm.data();
            if (cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) != cudaSuccess) st = GPE_ECUDA;
            if (st == GPE_OK) st = gpe_plan_create(&d, g->st, &g->plan);
            if (st == GPE_OK) st = plan_prepare(g->plan);
            if (st == GPE_OK && (cudaMalloc((void **)&g->d_ptrs, sizeof(void *) * d.batch) != cudaSuccess ||
                                 cudaMalloc((void **)&g->d_slots, sizeof(int) * d.batch) != cudaSuccess))
                st = GPE_ENOMEM;
            g->cap = d.batch;
            if (st == GPE_OK &&
                (cudaMallocHost((void **)&g->pin_out, sizeof(double) * 6 * (size_t)(2 * d.batch + 1)) != cudaSuccess ||
                 cudaMallocHost((void **)&g->pin_err, sizeof(int) * (size_t)(d.batch + 2)) != cudaSuccess))
                st = GPE_ENOMEM;
            for (int j = d.batch - 1; j >= 0; --j) g->free_slots.push_back(j);
            if (st != GPE_OK) {
                if (g->plan) gpe_plan_destroy(g->plan);
                if (g->st) cudaStreamDestroy(g->st);
                if (g->d_ptrs) cudaFree(g->d_ptrs);
                if (g->d_slots) cudaFree(g->d_slots);
                if (g->pin_out) cudaFreeHost(g->pin_out);
                if (g->pin_err) cudaFreeHost(g->pin_err);
                delete g;
                g = nullptr;
                std::lock_guard<std::mutex> lk(s->mu);
                s->used -= extra;
            } else {
                std::lock_guard<std::mutex> lk(s->mu);
                s->groups[r->key] = g;
            }
        }
        // state from the server's pool, ordered on the group stream: neither the
        // allocation nor the upload waits for the device (the pageable source
        // is staged by the driver before the call returns)
        if (st == GPE_OK && cudaMallocFromPoolAsync(&r->dpsi, r->psi_host.size(), s->pool, g->st) != cudaSuccess) {
            r->dpsi = nullptr;
            st = GPE_ENOMEM;
        }
        if (st == GPE_OK &&
            cudaMemcpyAsync(r->dpsi, r->psi_host.data(), r->psi_host.size(), cudaMemcpyHostToDevice, g->st) != cudaSuccess)
            st = GPE_ECUDA;
        if (st == GPE_OK) {
            r->slot = g->free_slots.back();
            g->free_slots.pop_back();
            st = plan_set_slot(g->plan, r->slot, r->r.desc.g, r->r.desc.gamma);
        }
        r->res.t_admit = now_s(s->t0);
        r->state = 1;
        if (st != GPE_OK) {
            finish_req(s, g, r, st);
            continue;
        }
        g->members.push_back(r);
    }
}

// upload the pointers and slots of `ms` to the group's device arrays
static bool upload_members(SGroup *g, const std::vector<Req *> &ms)
{
    std::vector<void *> hp(ms.size());
    std::vector<int> hs(ms.size());
    for (size_t j = 0; j < ms.size(); ++j) {
        hp[j] = ms[j]->dpsi;
        hs[j] = ms[j]->slot;
    }
    // pageable sources: staged by the driver before each call returns, so the
    // vectors may go out of scope; the copies stay ordered on the group stream
    return cudaMemcpyAsync(g->d_ptrs, hp.data(), sizeof(void *) * hp.size(), cudaMemcpyHostToDevice, g->st) == cudaSuccess &&
           cudaMemcpyAsync(g->d_slots, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice, g->st) == cudaSuccess;
}

// One scheduling round, in two phases.  First every group's work is
// enqueued on its own stream without waiting: real-time groups advance all
// members by one chunk (the smallest remaining step count, capped; chunking
// is exact); imaginary-time groups take the energy of new members' inputs,
// then advance sets of members with equal chunk, exactly min(check_every,
// remaining) steps between energy checks as gpe_step_imag does, each set's
// energies and error word copied into pinned buffers.  Then each stream is
// waited for once and the sets are retired in the order they were enqueued.
static void round_once(gpe_server *s)
{
    std::vector<SGroup *> gs;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &kv : s->groups)
            if (!kv.second->members.empty()) gs.push_back(kv.second);
    }
    struct Pending {
        SGroup *g;
        std::vector<Req *> ms;
        int64_t chunk;
        int kind;            // 0 real-time chunk, 1 imaginary-time set, 2 first energies
        double *o6;          // pinned energies, or NULL
        int *err;            // pinned error word, or NULL
        gpe_status st;       // enqueue status
    };
    std::vector<Pending> pend;
    for (SGroup *g : gs) {
        int used_sets = 0;
        size_t used_out = 0;
        auto land = [&](size_t count, double **o6, int **err) {
            *o6 = g->pin_out + 6 * used_out;
            used_out += count;
            *err = g->pin_err + used_sets;
            ++used_sets;
        };
        if (!g->imag) {
            int64_t chunk = s->chunk;
            for (Req *r : g->members) chunk = std::min(chunk, r->r.nsteps - r->done_steps);
            chunk = std::max<int64_t>(chunk, 1);
            gpe_status st = upload_members(g, g->members) ? GPE_OK : GPE_ECUDA;
            if (st == GPE_OK)
                st = plan_run(g->plan, 0, g->d_ptrs, g->d_slots, (int64_t)g->members.size(), chunk, 1.0, nullptr);
            // energies only when someone finishes (the report of the final state)
            bool need = false;
            for (Req *r : g->members) need = need || r->done_steps + chunk >= r->r.nsteps;
            double *o6 = nullptr;
            int *err = nullptr;
            if (st == GPE_OK && need) {
                land(g->members.size(), &o6, &err);
                st = plan_run_async(g->plan, 2, g->d_ptrs, g->d_slots, (int64_t)g->members.size(), 0, 1.0, o6, err);
            }
            pend.push_back({g, g->members, chunk, 0, o6, err, st});
            continue;
        }
        std::vector<Req *> fresh;
        for (Req *r : g->members)
            if (!r->has_e0) fresh.push_back(r);
        if (!fresh.empty()) {
            double *o6;
            int *err;
            land(fresh.size(), &o6, &err);
            gpe_status st = upload_members(g, fresh) ? GPE_OK : GPE_ECUDA;
            if (st == GPE_OK)
                st = plan_run_async(g->plan, 2, g->d_ptrs, g->d_slots, (int64_t)fresh.size(), 0, 1.0, o6, err);
            pend.push_back({g, fresh, 0, 2, o6, err, st});
        }
        std::map<int64_t, std::vector<Req *>> sets;
        for (Req *r : g->members)
            sets[std::min<int64_t>(r->r.check_every, r->r.nsteps - r->done_steps)].push_back(r);
        for (auto &kv : sets) {
            const int64_t chunk = std::max<int64_t>(kv.first, 1);
            double *o6;
            int *err;
            land(kv.second.size(), &o6, &err);
            gpe_status st = upload_members(g, kv.second) ? GPE_OK : GPE_ECUDA;
            if (st == GPE_OK)
                st = plan_run_async(g->plan, 1, g->d_ptrs, g->d_slots, (int64_t)kv.second.size(), chunk,
                                    kv.second[0]->r.target_norm, o6, err);
            pend.push_back({g, kv.second, chunk, 1, o6, err, st});
        }
    }
    std::map<SGroup *, gpe_status> synced;
    for (SGroup *g : gs) synced[g] = cudaStreamSynchronize(g->st) == cudaSuccess ? GPE_OK : GPE_ECUDA;
    for (Pending &pd : pend) {
        SGroup *g = pd.g;
        gpe_status st = pd.st != GPE_OK ? pd.st : synced[g];
        if (st == GPE_OK && pd.err && *pd.err)
            st = (*pd.err & (ERR_TMA_TIMEOUT | ERR_CLUSTER_TIMEOUT)) ? GPE_ETIMEOUT : GPE_ENUMERIC;
        if (pd.kind == 2) {
            for (size_t j = 0; j < pd.ms.size(); ++j) {
                Req *r = pd.ms[j];
                if (st != GPE_OK) {
                    finish_req(s, g, r, st);
                    g->members.erase(std::find(g->members.begin(), g->members.end(), r));
                    continue;
                }
                r->e_prev = pd.o6[6 * j + 4];
                r->has_e0 = true;
            }
            continue;
        }
        for (size_t j = 0; j < pd.ms.size(); ++j) {
            Req *r = pd.ms[j];
            if (std::find(g->members.begin(), g->members.end(), r) == g->members.end()) continue;   // retired earlier
            if (st == GPE_OK) r->done_steps += pd.chunk;
            if (pd.o6 && st == GPE_OK) {
                r->res.norm = pd.o6[6 * j + 0];
                r->res.energy = pd.o6[6 * j + 4];
            }
            bool finished = st != GPE_OK || r->done_steps >= r->r.nsteps;
            gpe_status rs = st;
            if (g->imag && st == GPE_OK) {
                if (!isfinite(r->res.energy)) {
                    rs = GPE_ENUMERIC;
                    finished = true;
                } else if (r->r.etol > 0.0 && fabs(r->res.energy - r->e_prev) < r->r.etol) {
                    finished = true;
                }
                r->e_prev = r->res.energy;
            }
            if (finished) {
                finish_req(s, g, r, rs);
                g->members.erase(std::find(g->members.begin(), g->members.end(), r));
            }
        }
    }
}

static void worker_main(gpe_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20),
                                [&] { return s->stop || !s->queue.empty() || s->active > 0; });
            if (s->stop) break;
        }
        admit(s);
        round_once(s);
    }
}

extern "C" gpe_status gpe_server_create(size_t hbm_budget_bytes, int max_active, int chunk_steps, gpe_server **out)
{
    if (!out || hbm_budget_bytes == 0) return sfail(GPE_EINVAL, "gpe_server_create: bad arguments");
    gpe_server *s = new gpe_server();
    s->budget = hbm_budget_bytes;
    // max_active <= 0: as many resident requests as the budget holds at 64 MiB
    // each (a 256^3 complex64 state is 128 MiB, a 1024^2 one 8 MiB), 16..256
    s->max_active = max_active > 0 ? max_active
                                   : (int)std::max<size_t>(16, std::min<size_t>(256, hbm_budget_bytes / (64ull << 20)));
    s->chunk = chunk_steps > 0 ? chunk_steps : 64;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return sfail(GPE_ECUDA, "cudaGetDevice failed");
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        delete s;
        return sfail(GPE_ECUDA, "cudaMemPoolCreate failed");
    }
    // keep freed states in the pool up to the budget instead of returning them
    cuuint64_t keep = (cuuint64_t)hbm_budget_bytes;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GPE_OK;
}

extern "C" gpe_status gpe_server_destroy(gpe_server *s)
{
    if (!s) return sfail(GPE_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    for (auto &kv : s->reqs) {
        if (kv.second->dpsi) cudaFree(kv.second->dpsi);
        delete kv.second;
    }
    for (auto &kv : s->groups) {
        SGroup *g = kv.second;
        if (g->plan) gpe_plan_destroy(g->plan);
        if (g->st) cudaStreamDestroy(g->st);
        if (g->d_ptrs) cudaFree(g->d_ptrs);
        if (g->d_slots) cudaFree(g->d_slots);
        if (g->pin_out) cudaFreeHost(g->pin_out);
        if (g->pin_err) cudaFreeHost(g->pin_err);
        delete g;
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return GPE_OK;
}

extern "C" gpe_status gpe_serve_submit(gpe_server *s, const gpe_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket || !req->psi0_host) return sfail(GPE_EINVAL, "gpe_serve_submit: NULL argument");
    gpe_status st = check_desc(req->desc);
    if (st != GPE_OK) return st;
    const gpe_plan_desc &d = req->desc;
    if (d.ndim < 1 || d.ndim > 3 || (d.prec != GPE_C64 && d.prec != GPE_C128))
        return sfail(GPE_EINVAL, "bad request description");
    if (req->nsteps < 1) return sfail(GPE_EINVAL, "nsteps must be >= 1");
    if (req->imag && (req->check_every < 1 || !(req->target_norm > 0.0)))
        return sfail(GPE_EINVAL, "imaginary-time requests need check_every >= 1 and target_norm > 0");
    int64_t N = 1;
    for (int a = 0; a < d.ndim; ++a) {
        if (d.n[a] < 2 || d.n[a] > 4096 || (d.n[a] & (d.n[a] - 1)))
            return sfail(GPE_EUNSUPPORTED, "each n[a] must be a power of two in [2, 4096]");
        N *= d.n[a];
    }
    Req *r = new Req();
    r->r = *req;
    r->r.psi0_host = nullptr;
    const size_t bytes = (size_t)N * (d.prec == GPE_C64 ? 8 : 16);
    r->psi_host.assign(static_cast<const unsigned char *>(req->psi0_host),
                       static_cast<const unsigned char *>(req->psi0_host) + bytes);
    r->bytes = bytes;
    r->key = group_key(d, req->imag ? 1 : 0);
    if (req->imag) {
        r->key.append(reinterpret_cast<const char *>(&req->target_norm), sizeof(double));
        r->key.append(reinterpret_cast<const char *>(&req->check_every), sizeof(int));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->res.t_submit = now_s(s->t0);
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
    s->cv_work.notify_all();
    return GPE_OK;
}

extern "C" gpe_status gpe_serve_poll(gpe_server *s, uint64_t ticket, int timeout_ms, gpe_result *res, void *psi_out_host)
{
    if (!s || !res) return sfail(GPE_EINVAL, "gpe_serve_poll: NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(GPE_EINVAL, "unknown ticket");
    Req *r = it->second;
    if (r->state != 2 && timeout_ms != 0) {
        auto pred = [&] { return r->state == 2; };
        if (timeout_ms < 0) s->cv_done.wait(lk, pred);
        else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    if (r->state != 2) return GPE_ENOTREADY;
    *res = r->res;
    if (psi_out_host && r->res.status == GPE_OK) memcpy(psi_out_host, r->psi_host.data(), r->psi_host.size());
    s->reqs.erase(it);
    delete r;
    return GPE_OK;
}

extern "C" gpe_status gpe_server_stats(gpe_server *s, int *queued, int *active, size_t *hbm_used)
{
    if (!s) return sfail(GPE_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->queue.size();
    if (active) *active = s->active;
    if (hbm_used) *hbm_used = s->used;
    return GPE_OK;
}
