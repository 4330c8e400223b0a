// server.cu -- continuous batching of encrypted matrix-product requests.
//
// Requests (two ciphertexts and a shape) are queued by hegmm_server_submit.
// hegmm_server_poll, called by the caller's event loop, (1) retires batches
// whose completion event has fired, releasing their workspace and recording
// each request's submit-to-completion latency, and (2) admits queued
// requests into a new batch whenever a device stream is free and the batch's
// estimated workspace fits in what the memory budget leaves.  A batch runs
// through the batch executor (one launch per stage over all of its
// products) on its own stream, so batches on different streams overlap on
// the device while new requests keep arriving.  Evaluation keys and plan
// masks stay resident in the context; every request's result is the same
// ciphertext it gives alone (the batch executor is bit-identical to the
// single-product path).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace hg {

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SrvReq {
    uint64_t id;
    const hegmm_ct *A, *B;
    int m, l, n, alg;
    double t_submit;
    size_t est;
};

struct SrvBatch {
    int stream;
    cudaEvent_t start, done;  // timed: the batch's first and last point on its stream
    std::vector<SrvReq> reqs;
    std::vector<hegmm_ct *> outs;
    std::vector<BatchPlan *> plans;  // one per algorithm group of the batch
    size_t bytes;
};

// A retired batch's device interval, in ms after the server's origin event.
struct SrvSpan {
    double t0, t1;
    int stream;
    bool overlapped;
};

struct SrvDone {
    hegmm_ct *C;
    double lat_ms;
    int rc;
};

}  // namespace hg

struct hegmm_server {
    hg::Ctx *c;
    hegmm_server_opts o;
    std::vector<cudaStream_t> streams;
    std::vector<int> busy;
    std::vector<char *> arena;  // per stream: workspace of its current batch
    size_t arena_cap = 0;
    cudaEvent_t inputs_ready = nullptr;
    cudaEvent_t origin = nullptr;  // timed, recorded at creation
    std::deque<hg::SrvSpan> spans;  // the most recent retired batches' intervals
    long long max_flight = 0, overlapped = 0;
    std::deque<hg::SrvReq> queue;
    std::vector<hg::SrvBatch> flight;
    std::map<uint64_t, hg::SrvDone> done;
    uint64_t next_id = 1;
    size_t inflight_bytes = 0;
    long long submitted = 0, completed = 0, batches = 0, failed = 0, max_batch_seen = 0;
    std::vector<double> lat;
};

using namespace hg;

// Retires finished batches; with block, waits for the oldest one.
static int retire(hegmm_server *s, bool block) {
    int n = 0;
    for (size_t i = 0; i < s->flight.size();) {
        SrvBatch &b = s->flight[i];
        cudaError_t q = (block && i == 0) ? cudaEventSynchronize(b.done) : cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) {
            i++;
            continue;
        }
        if (q != cudaSuccess) return cuda_check(s->c, "server batch");
        const double t = now_ms();
        // The batch's device interval, and whether it intersects that of
        // another stream's batch: both were then queued on the device at once.
        float a = 0.f, e = 0.f;
        if (cudaEventElapsedTime(&a, s->origin, b.start) == cudaSuccess &&
            cudaEventElapsedTime(&e, s->origin, b.done) == cudaSuccess) {
            SrvSpan sp{a, e, b.stream, false};
            for (SrvSpan &o : s->spans)
                if (o.stream != sp.stream && sp.t0 < o.t1 && o.t0 < sp.t1) {
                    if (!o.overlapped) s->overlapped++;
                    o.overlapped = true;
                    if (!sp.overlapped) s->overlapped++;
                    sp.overlapped = true;
                }
            s->spans.push_back(sp);
            if (s->spans.size() > 64) s->spans.pop_front();
        } else {
            cudaGetLastError();
        }
        for (size_t k = 0; k < b.reqs.size(); k++) {
            const double lm = t - b.reqs[k].t_submit;
            s->done[b.reqs[k].id] = {b.outs[k], lm, HEGMM_OK};
            s->lat.push_back(lm);
            s->completed++;
        }
        cudaStream_t old = s->c->st;
        s->c->st = s->streams[b.stream];
        for (BatchPlan *p : b.plans) release_plan(s->c, p);
        s->c->st = old;
        cudaEventDestroy(b.done);
        cudaEventDestroy(b.start);
        s->inflight_bytes -= b.bytes;
        s->busy[b.stream] = 0;
        s->flight.erase(s->flight.begin() + (long)i);
        n++;
        block = false;
    }
    return n;
}

// Admits queued requests into batches while streams and memory allow.
static int admit(hegmm_server *s) {
    Ctx *c = s->c;
    int launched = 0;
    while (!s->queue.empty()) {
        int st = -1;
        for (int i = 0; i < (int)s->streams.size(); i++)
            if (!s->busy[i]) {
                st = i;
                break;
            }
        if (st < 0) break;
        std::vector<SrvReq> reqs;
        size_t bytes = 2 * c->ws_budget;  // chunk scratch of one batch
        while (!s->queue.empty() && (int)reqs.size() < s->o.max_batch) {
            const SrvReq &r = s->queue.front();
            const bool fits = bytes + r.est <= s->arena_cap;  // the stream's arena
            if (!fits && !reqs.empty()) break;
            bytes += r.est;
            reqs.push_back(r);
            s->queue.pop_front();
        }
        if (reqs.empty()) break;
        std::vector<const hegmm_ct *> A, B;
        std::vector<int> mln;
        for (auto &r : reqs) {
            A.push_back(r.A);
            B.push_back(r.B);
            mln.insert(mln.end(), {r.m, r.l, r.n});
        }
        std::vector<hegmm_ct *> outs(reqs.size(), nullptr);
        cudaStream_t old = c->st;
        c->st = s->streams[st];
        c->arena = s->arena[st];
        c->arena_cap = s->arena_cap;
        c->arena_used = 0;
        cudaStreamWaitEvent(c->st, s->inputs_ready, 0);
        SrvBatch sb;
        cudaEventCreate(&sb.start);
        cudaEventRecord(sb.start, c->st);
        // one executor call for the whole batch; each request carries its
        // resolved algorithm
        std::vector<int> algs;
        for (auto &r : reqs) algs.push_back(r.alg);
        BatchPlan *plan = nullptr;
        std::vector<BatchPlan *> plans;
        int rc = matmul_run(c, (int)reqs.size(), A.data(), B.data(), mln.data(), HEGMM_ALG_AUTO, algs.data(),
                            outs.data(), nullptr, false, &plan);
        if (!rc) plans.push_back(plan);
        c->arena = nullptr;
        sb.stream = st;
        sb.bytes = bytes;
        cudaEventCreate(&sb.done);
        cudaEventRecord(sb.done, c->st);
        c->st = old;
        if (rc) {
            for (auto *p : plans) {
                c->st = s->streams[st];
                release_plan(c, p);
                c->st = old;
            }
            cudaEventDestroy(sb.done);
            cudaEventDestroy(sb.start);
            for (size_t k = 0; k < reqs.size(); k++) {
                hegmm_ct_destroy(outs[k]);
                s->done[reqs[k].id] = {nullptr, 0.0, rc};
                s->failed++;
            }
            continue;
        }
        sb.plans = plans;
        sb.reqs = reqs;
        sb.outs = outs;
        s->busy[st] = 1;
        s->inflight_bytes += bytes;
        s->batches++;
        s->max_batch_seen = std::max<long long>(s->max_batch_seen, (long long)reqs.size());
        s->flight.push_back(sb);
        s->max_flight = std::max<long long>(s->max_flight, (long long)s->flight.size());
        launched++;
    }
    return launched;
}

extern "C" {

int hegmm_server_create(hegmm_ctx *h, const hegmm_server_opts *opts, hegmm_server **out) {
    if (!h || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    hegmm_server *s = new hegmm_server;
    s->c = c;
    hegmm_server_opts o{64, 2, (uint64_t)16 << 30};
    if (opts) {
        if (opts->max_batch > 0) o.max_batch = opts->max_batch;
        if (opts->streams > 0) o.streams = std::min(opts->streams, 8);
        if (opts->mem_budget > 0) o.mem_budget = opts->mem_budget;
    }
    s->o = o;
    s->arena_cap = (size_t)(o.mem_budget / (uint64_t)o.streams) & ~(size_t)255;
    for (int i = 0; i < o.streams; i++) {
        cudaStream_t st = nullptr;
        void *a = nullptr;
        // arenas come from the context's stream-ordered pool, which also
        // holds what evicted masks and finished plans gave back
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            !(a = dalloc_evicting(c, s->arena_cap))) {
            cudaGetLastError();
            for (size_t k = 0; k < s->arena.size(); k++) cudaFreeAsync(s->arena[k], c->st);
            for (auto made : s->streams) cudaStreamDestroy(made);
            if (st) cudaStreamDestroy(st);
            delete s;
            return set_err(c, HEGMM_ENOMEM, "server streams / workspace");
        }
        s->streams.push_back(st);
        s->busy.push_back(0);
        s->arena.push_back((char *)a);
    }
    cudaEventCreateWithFlags(&s->inputs_ready, cudaEventDisableTiming);
    cudaEventCreate(&s->origin);
    cudaEventRecord(s->origin, c->st);
    cudaStreamSynchronize(c->st);  // keys and tables are complete before other streams use them
    *out = s;
    return cuda_check(c, "server create");
}

int hegmm_server_submit(hegmm_server *s, const hegmm_ct *A, const hegmm_ct *B, int m, int l, int n, int alg,
                        uint64_t *ticket) {
    if (!s || !A || !B || !ticket) return HEGMM_EINVAL;
    Ctx *c = s->c;
    if (alg < 0 || alg > 3) return set_err(c, HEGMM_EINVAL, "algorithm must be 0 (auto), 1, 2 or 3");
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    if (A->level != c->L || B->level != c->L) return set_err(c, HEGMM_EINVAL, "operand level does not match");
    SrvReq r{s->next_id++, A, B, m, l, n, a, now_ms(), estimate_bytes(c, m, l, n, a)};
    cudaEventRecord(s->inputs_ready, c->st);  // the operands were produced on the context stream
    s->queue.push_back(r);
    s->submitted++;
    *ticket = r.id;
    return cuda_check(c, "server submit");
}

int hegmm_server_poll(hegmm_server *s, int wait) {
    if (!s) return HEGMM_EINVAL;
    for (;;) {
        int r = retire(s, false);
        if (r < 0) return r;
        int a = admit(s);
        if (a < 0) return a;
        if (!wait) return HEGMM_OK;
        if (s->queue.empty() && s->flight.empty()) return HEGMM_OK;
        if (r == 0 && a == 0) {
            r = retire(s, true);
            if (r < 0) return r;
        }
    }
}

int hegmm_server_result(hegmm_server *s, uint64_t ticket, hegmm_ct **C, double *latency_ms) {
    if (!s || !C) return HEGMM_EINVAL;
    *C = nullptr;
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return HEGMM_OK;  // not finished yet
    const int rc = it->second.rc;
    *C = it->second.C;
    if (latency_ms) *latency_ms = it->second.lat_ms;
    s->done.erase(it);
    return rc;
}

int hegmm_server_stats_get(hegmm_server *s, hegmm_server_stats *st) {
    if (!s || !st) return HEGMM_EINVAL;
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->batches = s->batches;
    st->queued = (long long)s->queue.size();
    st->in_flight = 0;
    for (auto &b : s->flight) st->in_flight += (long long)b.reqs.size();
    st->max_batch = s->max_batch_seen;
    std::vector<double> v = s->lat;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * v.size() - 1 + 0.999999));
        return v[k];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_ms = v.empty() ? 0.0 : sum / v.size();
    st->max_ms = v.empty() ? 0.0 : v.back();
    st->max_batches_in_flight = s->max_flight;
    st->overlapped_batches = s->overlapped;
    return HEGMM_OK;
}

void hegmm_server_destroy(hegmm_server *s) {
    if (!s) return;
    hegmm_server_poll(s, 1);
    for (auto &kv : s->done) hegmm_ct_destroy(kv.second.C);
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (char *a : s->arena) cudaFreeAsync(a, s->c->st);
    cudaEventDestroy(s->inputs_ready);
    cudaEventDestroy(s->origin);
    delete s;
}

}  // extern "C"
