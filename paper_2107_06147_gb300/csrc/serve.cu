// serve.cu -- continuous batching of trajectory requests over libqtraj contexts (include/qtraj.h,
// "Serving").  Host code only: the device work of a launch is one qtraj_evolve (fused form) plus an
// asynchronous copy of its records to a pinned buffer, followed by an event that qtraj_poll queries.
// Nothing here waits for the device except qtraj_server_create and qtraj_server_destroy.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "api_internal.h"
#include "qtraj.h"

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

qtraj_status failf(qtraj_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
qtraj_status failf(qtraj_status st, const char *fmt, ...)
{
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    return qt::api_fail(st, b);
}

#define SCK(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return failf(QTRAJ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)
#define SOK(call)                                                                                          \
    do {                                                                                                   \
        qtraj_status s_ = (call);                                                                          \
        if (s_ != QTRAJ_OK) return s_;                                                                     \
    } while (0)

struct Request {
    uint64_t id;
    std::vector<qtraj_traj_desc> desc;
    std::vector<qtraj_obs> out;
    int remaining = 0;
    double work = 0.0;    // sum over its trajectories of N log2 N x steps (the order QTRAJ_ORDER_SHORTEST)
    uint64_t seq = 0;     // arrival order
};

// the trajectories of one request with one grid size, handed out in order
struct PendingPart {
    uint64_t id;
    std::vector<int> idx;
    size_t next = 0;
    double work = 0.0;    // of its request
    uint64_t seq = 0;
};

// a run of consecutive trajectories of a launch: request id, its descriptor positions idx
struct LaunchPart {
    uint64_t id;
    std::vector<int> idx;
};

struct Slot {
    qtraj_ctx *ctx = nullptr;
    int N = 0, cap = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t_start = nullptr, t_end = nullptr;   // timing events around a launch's evolve
    int launch_traj = 0;
    qtraj_obs *h_obs = nullptr;
    bool busy = false;
    std::vector<LaunchPart> parts;
    // per-launch host arrays (kept so that no launch allocates on the host either, once warm)
    std::vector<int> spec_idx, medium_idx;
    std::vector<uint64_t> seeds;
    std::vector<qtraj_medium> media;
};

struct PerN {
    int N = 0, cap = 0;
    std::vector<Slot> slots;
    std::deque<PendingPart> pending;   // arrival order; QTRAJ_ORDER_SHORTEST picks the least work first
};

bool valid_n(int N) { return N >= 16 && N <= 16384 && (N & (N - 1)) == 0; }

qtraj_status check_config(const qtraj_server_config *c)
{
    if (!c || !c->Ns || !c->params || !c->specs) return failf(QTRAJ_EINVAL, "null argument");
    if (c->n_N <= 0) return failf(QTRAJ_EINVAL, "n_N must be positive");
    for (int i = 0; i < c->n_N; ++i) {
        if (!valid_n(c->Ns[i])) return failf(QTRAJ_EINVAL, "grid size %d: a power of two in [16, 16384]", c->Ns[i]);
        for (int k = 0; k < i; ++k)
            if (c->Ns[k] == c->Ns[i]) return failf(QTRAJ_EINVAL, "grid size %d listed twice", c->Ns[i]);
    }
    if (!(c->dr > 0) || !(c->dt > 0) || !(c->M > 0)) return failf(QTRAJ_EINVAL, "dr, dt, M must be positive");
    if (c->n_specs <= 0 || c->n_specs > QTRAJ_SERVER_MAX_SPECS)
        return failf(QTRAJ_EINVAL, "n_specs must be in [1, %d]", QTRAJ_SERVER_MAX_SPECS);
    if (c->slots_per_n <= 0 || c->waves_per_launch <= 0 || c->max_inflight_traj <= 0)
        return failf(QTRAJ_EINVAL, "slots_per_n, waves_per_launch and max_inflight_traj must be positive");
    if (c->order != QTRAJ_ORDER_ARRIVAL && c->order != QTRAJ_ORDER_SHORTEST)
        return failf(QTRAJ_EINVAL, "order must be QTRAJ_ORDER_ARRIVAL or QTRAJ_ORDER_SHORTEST");
    return QTRAJ_OK;
}

qtraj_params slot_params(const qtraj_server_config *c)
{
    qtraj_params p = *c->params;
    p.form = QTRAJ_FUSED;
    p.save_states = 0;
    p.use_rmin = 0;
    return p;
}

// trajectories per launch of grid size N: waves x (SMs x resident CTAs of the fused kernel)
qtraj_status capacity_of(const qtraj_server_config *c, int N, int *cap)
{
    qtraj_params p = slot_params(c);
    qtraj_ctx *ctx = nullptr;
    SOK(qtraj_create(N, N * c->dr, c->dt, c->M, &p, &ctx));
    qtraj_kernel_info ki{};
    const qtraj_status st = qtraj_kernel_info_get(ctx, &ki);
    if (st == QTRAJ_OK) *cap = c->waves_per_launch * ki.sm_count * ki.ctas_per_sm;
    qtraj_destroy(ctx);
    return st;
}

} // namespace

struct qtraj_server {
    qtraj_server_config cfg{};
    std::vector<int> Ns;
    qtraj_params params{};
    std::vector<qtraj_init_spec> specs;
    std::vector<PerN> perN;                      // in the order of cfg.Ns
    std::map<int, int> n_index;                  // N -> index into perN
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<uint64_t> waiting;                // submitted, not admitted
    std::deque<uint64_t> done;                   // finished, not yet reported by qtraj_poll
    int64_t inflight = 0;                        // trajectories of admitted, unreturned requests
    int admitted = 0;
    uint64_t seq = 0;                            // arrival counter
    cudaEvent_t epoch = nullptr;                 // recorded at creation: the zero of the launch log
    std::vector<qtraj_launch_rec> log;           // finished launches
};

extern "C" {

qtraj_status qtraj_server_workspace_bytes(const qtraj_server_config *cfg, size_t *bytes)
{
    qt::api_clear_error();
    if (!bytes) return failf(QTRAJ_EINVAL, "null argument");
    SOK(check_config(cfg));
    qtraj_params p = slot_params(cfg);
    size_t total = 0;
    for (int i = 0; i < cfg->n_N; ++i) {
        const int N = cfg->Ns[i];
        int cap = 0;
        SOK(capacity_of(cfg, N, &cap));
        qtraj_ctx *ctx = nullptr;
        SOK(qtraj_create(N, N * cfg->dr, cfg->dt, cfg->M, &p, &ctx));
        const size_t b = qtraj_workspace_bytes(ctx, cap);
        qtraj_destroy(ctx);
        total += (size_t)cfg->slots_per_n * align256(b);
    }
    *bytes = total;
    return QTRAJ_OK;
}

qtraj_status qtraj_server_create(const qtraj_server_config *cfg, void *d_ws, size_t bytes, qtraj_server **out)
{
    qt::api_clear_error();
    if (!out || !d_ws) return failf(QTRAJ_EINVAL, "null argument");
    *out = nullptr;
    SOK(check_config(cfg));
    if (((uintptr_t)d_ws & 255) != 0) return failf(QTRAJ_EINVAL, "workspace must be 256-byte aligned");
    size_t need = 0;
    SOK(qtraj_server_workspace_bytes(cfg, &need));
    if (bytes < need) return failf(QTRAJ_ENOMEM, "workspace of %zu bytes < %zu required", bytes, need);

    std::unique_ptr<qtraj_server> s(new qtraj_server);
    s->cfg = *cfg;
    s->Ns.assign(cfg->Ns, cfg->Ns + cfg->n_N);
    s->cfg.Ns = s->Ns.data();
    s->params = slot_params(cfg);
    s->cfg.params = &s->params;
    s->specs.assign(cfg->specs, cfg->specs + cfg->n_specs);
    s->cfg.specs = s->specs.data();
    s->perN.resize(cfg->n_N);
    char *ws = (char *)d_ws;
    qtraj_status st = QTRAJ_OK;
    for (int i = 0; i < cfg->n_N && st == QTRAJ_OK; ++i) {
        PerN &pn = s->perN[i];
        pn.N = cfg->Ns[i];
        s->n_index[pn.N] = i;
        if ((st = capacity_of(cfg, pn.N, &pn.cap)) != QTRAJ_OK) break;
        pn.slots.resize(cfg->slots_per_n);
        for (Slot &sl : pn.slots) {
            sl.N = pn.N;
            sl.cap = pn.cap;
            if ((st = qtraj_create(pn.N, pn.N * cfg->dr, cfg->dt, cfg->M, &s->params, &sl.ctx)) != QTRAJ_OK) break;
            const size_t b = align256(qtraj_workspace_bytes(sl.ctx, pn.cap));
            std::vector<int> zero(pn.cap, 0);
            if ((st = qtraj_init(sl.ctx, ws, b, pn.cap, s->specs.data(), cfg->n_specs, zero.data())) != QTRAJ_OK) break;
            ws += b;
            if ((st = qt::reserve_media(sl.ctx, pn.cap)) != QTRAJ_OK) break;
            if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreate(&sl.t_start) != cudaSuccess || cudaEventCreate(&sl.t_end) != cudaSuccess ||
                cudaMallocHost(&sl.h_obs, sizeof(qtraj_obs) * pn.cap) != cudaSuccess) {
                st = failf(QTRAJ_ECUDA, "stream, event or pinned buffer: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            sl.spec_idx.reserve(pn.cap);
            sl.medium_idx.reserve(pn.cap);
            sl.seeds.reserve(pn.cap);
            sl.media.reserve(pn.cap);
        }
    }
    if (st == QTRAJ_OK && (cudaEventCreate(&s->epoch) != cudaSuccess || cudaEventRecord(s->epoch, 0) != cudaSuccess ||
                           cudaEventSynchronize(s->epoch) != cudaSuccess))
        st = failf(QTRAJ_ECUDA, "epoch event: %s", cudaGetErrorString(cudaGetLastError()));
    if (st != QTRAJ_OK) {
        qtraj_server_destroy(s.release());
        return st;
    }
    *out = s.release();
    return QTRAJ_OK;
}

qtraj_status qtraj_submit(qtraj_server *s, const qtraj_traj_desc *traj, int n, uint64_t request_id)
{
    qt::api_clear_error();
    if (!s || !traj) return failf(QTRAJ_EINVAL, "null argument");
    if (n <= 0) return failf(QTRAJ_EINVAL, "n must be positive");
    if (s->reqs.count(request_id)) return failf(QTRAJ_EINVAL, "request id %llu is queued or not yet returned",
                                                (unsigned long long)request_id);
    for (int t = 0; t < n; ++t) {
        if (!s->n_index.count(traj[t].N)) return failf(QTRAJ_EINVAL, "trajectory %d: grid size %d not served", t, traj[t].N);
        if (traj[t].spec < 0 || traj[t].spec >= (int)s->specs.size())
            return failf(QTRAJ_EINVAL, "trajectory %d: spec %d outside the catalogue", t, traj[t].spec);
        if (const char *why = qt::medium_problem(traj[t].medium)) return failf(QTRAJ_EINVAL, "trajectory %d: %s", t, why);
    }
    std::unique_ptr<Request> r(new Request);
    r->id = request_id;
    r->desc.assign(traj, traj + n);
    r->out.assign(n, qtraj_obs{});
    r->remaining = n;
    r->seq = s->seq++;
    for (int t = 0; t < n; ++t) {
        const qtraj_medium &m = traj[t].medium;
        // the Bjorken medium's steps, as the engine counts them (work estimate only)
        const double tau_f = m.tau0 * std::pow(m.T0 / m.Tf, 3.0);
        const double steps = m.T0 > m.Tf ? std::ceil((tau_f - m.tau0) / (0.1973269804 * s->cfg.dt)) : 0.0;
        r->work += (double)traj[t].N * std::log2((double)traj[t].N) * steps;
    }
    s->reqs[request_id] = std::move(r);
    s->waiting.push_back(request_id);
    return QTRAJ_OK;
}

namespace {

// moves the records of a finished launch into their requests
void collect(qtraj_server *s, Slot &sl)
{
    qtraj_launch_rec rec{sl.N, sl.launch_traj, (int)sl.parts.size(), 0, -1.0, -1.0};
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, s->epoch, sl.t_start) == cudaSuccess &&
        cudaEventElapsedTime(&b, s->epoch, sl.t_end) == cudaSuccess) {
        rec.start_ms = a;
        rec.end_ms = b;
    }
    s->log.push_back(rec);
    int o = 0;
    for (LaunchPart &p : sl.parts) {
        Request &r = *s->reqs.at(p.id);
        for (int k : p.idx) r.out[k] = sl.h_obs[o++];
        r.remaining -= (int)p.idx.size();
        if (r.remaining == 0) {
            s->done.push_back(r.id);
            --s->admitted;
        }
    }
    sl.parts.clear();
    sl.busy = false;
}

void admit(qtraj_server *s)
{
    while (!s->waiting.empty()) {
        Request &r = *s->reqs.at(s->waiting.front());
        const int64_t n = (int64_t)r.desc.size();
        if (s->inflight + n > s->cfg.max_inflight_traj && s->inflight > 0) break;
        s->waiting.pop_front();
        s->inflight += n;
        ++s->admitted;
        // split by grid size, keeping submission order inside each
        std::map<int, std::vector<int>> byN;
        for (int t = 0; t < (int)n; ++t) byN[r.desc[t].N].push_back(t);
        for (auto &kv : byN)
            s->perN[s->n_index.at(kv.first)].pending.push_back(PendingPart{r.id, std::move(kv.second), 0, r.work, r.seq});
    }
}

qtraj_status launch(qtraj_server *s, PerN &pn, Slot &sl)
{
    sl.spec_idx.clear();
    sl.medium_idx.clear();
    sl.seeds.clear();
    sl.media.clear();
    sl.parts.clear();
    std::map<std::tuple<double, double, double, double, double>, int> mkey;
    int n = 0;
    while (!pn.pending.empty() && n < sl.cap) {
        // the next part: the front (arrival order), or the one of least work
        auto it_pp = pn.pending.begin();
        if (s->cfg.order == QTRAJ_ORDER_SHORTEST)
            for (auto i2 = pn.pending.begin(); i2 != pn.pending.end(); ++i2)
                if (i2->work < it_pp->work || (i2->work == it_pp->work && i2->seq < it_pp->seq)) it_pp = i2;
        PendingPart &pp = *it_pp;
        const Request &r = *s->reqs.at(pp.id);
        LaunchPart lp{pp.id, {}};
        while (pp.next < pp.idx.size() && n < sl.cap) {
            const int k = pp.idx[pp.next++];
            const qtraj_traj_desc &d = r.desc[k];
            const auto key = std::make_tuple(d.medium.T0, d.medium.tau0, d.medium.Tf, d.medium.kappa_hat, d.medium.gamma_hat);
            auto it = mkey.find(key);
            int mi;
            if (it == mkey.end()) {
                mi = (int)sl.media.size();
                mkey.emplace(key, mi);
                sl.media.push_back(d.medium);
            } else {
                mi = it->second;
            }
            sl.spec_idx.push_back(d.spec);
            sl.medium_idx.push_back(mi);
            sl.seeds.push_back(d.seed);
            lp.idx.push_back(k);
            ++n;
        }
        sl.parts.push_back(std::move(lp));
        if (pp.next == pp.idx.size()) pn.pending.erase(it_pp);
    }
    if (n == 0) return QTRAJ_OK;
    SOK(qtraj_set_spec_idx(sl.ctx, sl.spec_idx.data(), n));
    SCK(cudaEventRecord(sl.t_start, sl.stream));
    SOK(qtraj_evolve(sl.ctx, n, sl.media.data(), (int)sl.media.size(), sl.medium_idx.data(), sl.seeds.data(),
                     (void *)sl.stream));
    SCK(cudaEventRecord(sl.t_end, sl.stream));
    SOK(qt::obs_to_host_async(sl.ctx, sl.h_obs, sl.stream));
    SCK(cudaEventRecord(sl.done, sl.stream));
    sl.launch_traj = n;
    sl.busy = true;
    return QTRAJ_OK;
}

} // namespace

qtraj_status qtraj_poll(qtraj_server *s, uint64_t *done_ids, int capacity, int *n_done)
{
    qt::api_clear_error();
    if (!s || !n_done || (capacity > 0 && !done_ids) || capacity < 0) return failf(QTRAJ_EINVAL, "bad argument");
    *n_done = 0;
    for (PerN &pn : s->perN)
        for (Slot &sl : pn.slots) {
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) return failf(QTRAJ_ECUDA, "launch on N=%d failed: %s", sl.N, cudaGetErrorString(e));
            collect(s, sl);
        }
    admit(s);
    for (PerN &pn : s->perN)
        for (Slot &sl : pn.slots)
            if (!sl.busy && !pn.pending.empty()) SOK(launch(s, pn, sl));
    while (*n_done < capacity && !s->done.empty()) {
        done_ids[(*n_done)++] = s->done.front();
        s->done.pop_front();
    }
    return QTRAJ_OK;
}

qtraj_status qtraj_request_result(qtraj_server *s, uint64_t request_id, qtraj_obs *out, int n)
{
    qt::api_clear_error();
    if (!s || !out) return failf(QTRAJ_EINVAL, "null argument");
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return failf(QTRAJ_EINVAL, "unknown request id %llu", (unsigned long long)request_id);
    Request &r = *it->second;
    if (r.remaining > 0) return failf(QTRAJ_EBUSY, "request %llu has %d trajectories outstanding",
                                      (unsigned long long)request_id, r.remaining);
    if (n != (int)r.out.size()) return failf(QTRAJ_EINVAL, "request %llu has %zu records, not %d",
                                             (unsigned long long)request_id, r.out.size(), n);
    for (uint64_t d : s->done)
        if (d == request_id) return failf(QTRAJ_EINVAL, "request %llu has not been reported by qtraj_poll yet",
                                          (unsigned long long)request_id);
    std::memcpy(out, r.out.data(), sizeof(qtraj_obs) * n);
    s->inflight -= n;
    s->reqs.erase(it);
    return QTRAJ_OK;
}

qtraj_status qtraj_server_counts(const qtraj_server *s, int *waiting, int *admitted, int *launches_in_flight)
{
    qt::api_clear_error();
    if (!s) return failf(QTRAJ_EINVAL, "null argument");
    int busy = 0;
    for (const PerN &pn : s->perN)
        for (const Slot &sl : pn.slots) busy += sl.busy;
    if (waiting) *waiting = (int)s->waiting.size();
    if (admitted) *admitted = s->admitted;
    if (launches_in_flight) *launches_in_flight = busy;
    return QTRAJ_OK;
}

qtraj_status qtraj_server_launch_log(qtraj_server *s, qtraj_launch_rec *out, int capacity, int *n_written, int clear)
{
    qt::api_clear_error();
    if (!s || !n_written || capacity < 0 || (capacity > 0 && !out)) return failf(QTRAJ_EINVAL, "bad argument");
    const int n = (int)std::min<size_t>((size_t)capacity, s->log.size());
    if (n) std::memcpy(out, s->log.data(), sizeof(qtraj_launch_rec) * n);
    *n_written = n;
    if (clear) s->log.clear();
    return QTRAJ_OK;
}

void qtraj_server_destroy(qtraj_server *s)
{
    if (!s) return;
    for (PerN &pn : s->perN)
        for (Slot &sl : pn.slots) {
            if (sl.stream) cudaStreamSynchronize(sl.stream);
            if (sl.ctx) qtraj_destroy(sl.ctx);
            if (sl.h_obs) cudaFreeHost(sl.h_obs);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.t_start) cudaEventDestroy(sl.t_start);
            if (sl.t_end) cudaEventDestroy(sl.t_end);
            if (sl.stream) cudaStreamDestroy(sl.stream);
        }
    if (s->epoch) cudaEventDestroy(s->epoch);
    delete s;
}

} // extern "C"
