// Serving form: continuous batching of eigenproblems of mixed orders.
//
// Requests arrive through pjac_serve_submit (host buffers).  The scheduler
// runs from submit, poll and progress (no background thread).  Its admission
// policy (serve_sched.h): small requests (order <= 256) first, as
// micro-batches on the batched kernels; otherwise the oldest large request
// alone on the single-problem path (cluster-parallel Jacobi), while the SMs
// of all running large requests fit outside a reserve of one eighth of the
// device; the oldest large request is passed over by at most four
// micro-batches.
// Each lane has its own solver handle and one CUDA stream.  An eighth of the
// lanes (at least one, from two lanes up) have a stream at the device's
// highest priority and take only micro-batches, which go to them first; the
// others have one at its lowest.  One Jacobi CTA fills an SM's register file, so without the
// reserve the large solves would hold every SM for seconds and a small
// request would wait behind them; with it, small work always finds SMs, and
// the stream priority puts its CTAs ahead of queued low-priority ones.
// Streams beyond CUDA_DEVICE_MAX_CONNECTIONS share hardware queues, in which
// work runs in submission order: a micro-batch could then wait behind a
// large solve of another lane.  Hence one stream per lane, and the advice to
// raise that limit to 32 and keep max_slots <= 32.
// Creating a server loads all kernels of the library on the current device,
// so that no first-launch load happens while requests run.
// A lane's results are copied back on its stream; completion is detected
// with an event query, and the lane is recycled at once.
// Latency = completion detected - submit.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>
#include "internal.h"
#include "serve_sched.h"

namespace pjac {
int set_err(int code, const char* fmt, ...);
int cuda_err(cudaError_t e, const char* what);
}
using namespace pjac;

namespace {

using clk = std::chrono::steady_clock;

double now_ms() {
    return std::chrono::duration<double, std::milli>(clk::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    int n;
    pjac_pivot pivot;
    double tol;
    std::vector<double> a;       // host copy of A (column-major, ld n)
    double* w_out;
    double* v_out;
    int ldv;
    double t_submit;
    double t_done;
    int status = PJAC_PENDING;
    pjac_info info;
    size_t footprint;
    int bypassed = 0;            // micro-batches admitted ahead of it while it could have run
};

struct Lane {
    cudaStream_t st = nullptr;
    bool hi = false;                 // high-priority stream: micro-batches only
    int sms = 0;                     // SMs held by the current large request, 0 for a micro-batch
    pjac_handle* h = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request*> reqs;
    // device buffers (grown on demand) and pinned host staging
    double* dA = nullptr; size_t dA_bytes = 0;
    double* dW = nullptr; size_t dW_bytes = 0;
    double* dV = nullptr; size_t dV_bytes = 0;
    pjac_info* dInfo = nullptr; size_t dInfo_bytes = 0;
    double* hA = nullptr; size_t hA_bytes = 0;
    double* hW = nullptr; size_t hW_bytes = 0;
    double* hV = nullptr; size_t hV_bytes = 0;
    pjac_info* hInfo = nullptr; size_t hInfo_bytes = 0;
    std::vector<int> ns;
    std::vector<int64_t> aoff, woff;
    std::vector<void*> retired;   // outgrown pinned buffers, freed when the server is destroyed
    size_t footprint = 0;
    int launch_status = PJAC_OK;
};

// Lane buffers grow to the next power of two, stream-ordered on the lane's
// stream (device) so that growing never waits for other lanes' work.
size_t pow2_at_least(size_t x) {
    size_t p = 4096;
    while (p < x) p <<= 1;
    return p;
}

template <class T>
int grow_dev(T*& p, size_t& cur, size_t need, cudaStream_t st) {
    if (need <= cur) return PJAC_OK;
    need = pow2_at_least(need);
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    cur = 0;
    cudaError_t e = cudaMallocAsync((void**)&p, need, st);
    if (e != cudaSuccess) { cudaGetLastError(); return set_err(PJAC_ENOMEM, "serve: cudaMalloc %zu", need); }
    cur = need;
    return PJAC_OK;
}

// Pinned host buffers are never freed while the server runs (cudaFreeHost
// waits for the whole device): an outgrown one is retired.
template <class T>
int grow_host(T*& p, size_t& cur, size_t need, std::vector<void*>& retired) {
    if (need <= cur) return PJAC_OK;
    need = pow2_at_least(need);
    if (p) retired.push_back(p);
    p = nullptr;
    cur = 0;
    cudaError_t e = cudaMallocHost((void**)&p, need);
    if (e != cudaSuccess) { cudaGetLastError(); return set_err(PJAC_ENOMEM, "serve: cudaMallocHost %zu", need); }
    cur = need;
    return PJAC_OK;
}

// Device bytes a request holds while admitted: input, outputs and the
// solver's workspace (about 4 n^2 doubles plus FP32 state).
size_t request_footprint(int n) {
    size_t nn = (size_t)n * n;
    return nn * 8 * 7 + nn * 4 * 6 + (size_t)n * 64 + 4096;
}

}  // namespace

struct pjac_server {
    pjac_serve_opts o;
    std::mutex mu;
    std::vector<Lane> lanes;
    ServeQueue<Request> q;                       // waiting requests, admitted bytes and SMs
    std::unordered_map<uint64_t, Request*> all;   // queued, running or finished-not-polled
    uint64_t next_ticket = 1;
    int64_t inflight = 0, peak_inflight = 0;
    size_t peak_hbm = 0;
    int64_t launches = 0;                        // kernel launches of this library enqueued so far
    std::vector<double> lat_ms;
    double first_submit = -1, last_done = -1;
};

extern "C" void pjac_serve_default_opts(pjac_serve_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->max_slots = 8;
    o->max_queue = 1 << 16;
    o->hbm_budget_bytes = (size_t)8 << 30;
    pjac_default_opts(&o->solver);
}

extern "C" int pjac_serve_create(pjac_server** s, const pjac_serve_opts* o) {
    if (!s) return set_err(PJAC_EINVAL, "s is NULL");
    *s = nullptr;
    pjac_serve_opts d;
    pjac_serve_default_opts(&d);
    if (o) {
        d = *o;
        if (d.max_slots <= 0) d.max_slots = 8;
        if (d.max_queue <= 0) d.max_queue = 1 << 16;
        if (d.hbm_budget_bytes == 0) d.hbm_budget_bytes = (size_t)8 << 30;
    }
    if (d.max_slots > 64) return set_err(PJAC_EINVAL, "max_slots must be <= 64");
    auto* sv = new pjac_server();
    sv->o = d;
    int dev = 0, sms = 0, prio_lo = 0, prio_hi = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess || cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return set_err(PJAC_ECUDA, "serve: device query failed");
    }
    sv->q.sms_cap = sms - sms / 8;
    sv->q.budget = d.hbm_budget_bytes;
    // Load every kernel now: under lazy module loading a kernel's first
    // launch loads it, and the load can wait for work already running on the
    // device, which would stall the scheduler behind seconds-long solves.
    cudaError_t el = preload_batched_kernels();
    if (el == cudaSuccess) el = preload_diag32_kernels();
    if (el == cudaSuccess) el = preload_gemm_kernels();
    if (el == cudaSuccess) el = preload_tc_kernels();
    if (el == cudaSuccess) el = preload_jacobi_kernels();
    if (el == cudaSuccess) el = preload_svd_kernels();
    if (el == cudaSuccess) el = preload_os_kernels();
    if (el == cudaSuccess) el = preload_multi_kernels();
    if (el != cudaSuccess) {
        delete sv;
        return cuda_err(el, "serve: loading the kernels");
    }
    sv->lanes.resize(d.max_slots);
    int n_hi = d.max_slots >= 2 ? std::max(1, d.max_slots / 8) : 0;
    for (int li = 0; li < d.max_slots; ++li) {
        Lane& L = sv->lanes[li];
        L.hi = li < n_hi;
        // no autotuning on the lanes: a request's result must not depend on
        // which micro-batch (and which tuning state) it lands in
        pjac_opts lo = d.solver;
        lo.autotune = 0;
        int r = pjac_create(&L.h, &lo);
        // a served request's preconditioner must start beside running solves:
        // its cooperative kernels use at most 64 CTAs instead of the whole GPU
        if (r == PJAC_OK) handle_set_coop_cap(L.h, 64);
        cudaError_t e1 = cudaStreamCreateWithPriority(&L.st, cudaStreamNonBlocking, L.hi ? prio_hi : prio_lo);
        cudaError_t e2 = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (r != PJAC_OK || e1 != cudaSuccess || e2 != cudaSuccess) {
            pjac_serve_destroy(sv);
            return r != PJAC_OK ? r : set_err(PJAC_ECUDA, "serve: stream/event creation failed");
        }
    }
    *s = sv;
    return PJAC_OK;
}

extern "C" int pjac_serve_destroy(pjac_server* s) {
    if (!s) return PJAC_OK;
    for (auto& L : s->lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
    }
    for (auto& L : s->lanes) {
        if (L.h) pjac_destroy(L.h);
        if (L.st) cudaStreamDestroy(L.st);
        if (L.done) cudaEventDestroy(L.done);
        cudaFree(L.dA); cudaFree(L.dW); cudaFree(L.dV); cudaFree(L.dInfo);
        cudaFreeHost(L.hA); cudaFreeHost(L.hW); cudaFreeHost(L.hV); cudaFreeHost(L.hInfo);
        for (void* q : L.retired) cudaFreeHost(q);
    }
    for (auto& kv : s->all) delete kv.second;
    delete s;
    return PJAC_OK;
}

// Enqueue the work of a lane (its requests are already chosen).
static int launch_lane(pjac_server* s, Lane& L) {
    int nb = (int)L.reqs.size();
    size_t totA = 0, totW = 0;
    L.ns.resize(nb); L.aoff.resize(nb); L.woff.resize(nb);
    for (int k = 0; k < nb; ++k) {
        int n = L.reqs[k]->n;
        L.ns[k] = n;
        L.aoff[k] = (int64_t)totA;
        L.woff[k] = (int64_t)totW;
        totA += (size_t)n * n;
        totW += (size_t)n;
    }
    int r = PJAC_OK;
    if ((r = grow_dev(L.dA, L.dA_bytes, totA * 8, L.st))) return r;
    if ((r = grow_dev(L.dV, L.dV_bytes, totA * 8, L.st))) return r;
    if ((r = grow_dev(L.dW, L.dW_bytes, totW * 8, L.st))) return r;
    if ((r = grow_dev(L.dInfo, L.dInfo_bytes, sizeof(pjac_info) * nb, L.st))) return r;
    if ((r = grow_host(L.hA, L.hA_bytes, totA * 8, L.retired))) return r;
    if ((r = grow_host(L.hV, L.hV_bytes, totA * 8, L.retired))) return r;
    if ((r = grow_host(L.hW, L.hW_bytes, totW * 8, L.retired))) return r;
    if ((r = grow_host(L.hInfo, L.hInfo_bytes, sizeof(pjac_info) * nb, L.retired))) return r;
    for (int k = 0; k < nb; ++k)
        memcpy(L.hA + L.aoff[k], L.reqs[k]->a.data(), (size_t)L.ns[k] * L.ns[k] * 8);
    cudaError_t e = cudaMemcpyAsync(L.dA, L.hA, totA * 8, cudaMemcpyHostToDevice, L.st);
    if (e != cudaSuccess) return cuda_err(e, "serve H2D");
    Request* r0 = L.reqs[0];
    bool batched = r0->n <= SERVE_BATCH_MAX_N;
    if (batched) {
        r = pjac_solve_batched(L.h, nb, L.ns.data(), L.aoff.data(), L.dA, L.woff.data(), L.dW, L.aoff.data(),
                               L.dV, r0->pivot, r0->tol, L.dInfo, L.st);
        if (r == PJAC_OK) s->launches += batched_launch_count(s->o.solver.no_precondition);
    } else {
        // single large request: asynchronous single-problem path
        r = solve_async_dev(L.h, L.dA, r0->n, r0->n, r0->pivot, r0->tol, L.dW, L.dV, r0->n, L.dInfo, L.st);
        // as many as pjac_solve: no device input check (the host checked at
        // submission), one kernel more to copy the report
        if (r == PJAC_OK) s->launches += pjac_solve_launch_count(L.h, r0->n);
    }
    if (r != PJAC_OK) return r;
    e = cudaMemcpyAsync(L.hW, L.dW, totW * 8, cudaMemcpyDeviceToHost, L.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.hV, L.dV, totA * 8, cudaMemcpyDeviceToHost, L.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.hInfo, L.dInfo, sizeof(pjac_info) * nb, cudaMemcpyDeviceToHost, L.st);
    if (e == cudaSuccess) e = cudaEventRecord(L.done, L.st);
    if (e != cudaSuccess) return cuda_err(e, "serve D2H");
    return PJAC_OK;
}

static void finish_lane(pjac_server* s, Lane& L, int launch_err) {
    double t = now_ms();
    for (size_t k = 0; k < L.reqs.size(); ++k) {
        Request* q = L.reqs[k];
        if (launch_err != PJAC_OK) {
            q->status = launch_err;
            memset(&q->info, 0, sizeof(q->info));
            q->info.status = launch_err;
            q->info.n = q->n;
        } else {
            int n = q->n;
            memcpy(q->w_out, L.hW + L.woff[k], (size_t)n * 8);
            if (q->v_out)
                for (int c = 0; c < n; ++c)
                    memcpy(q->v_out + (size_t)c * q->ldv, L.hV + L.aoff[k] + (size_t)c * n, (size_t)n * 8);
            q->info = L.hInfo[k];
            q->status = q->info.status;
        }
        q->t_done = t;
        s->lat_ms.push_back(t - q->t_submit);
        s->last_done = t;
        s->inflight--;
    }
    serve_release(s->q, L);
    L.reqs.clear();
    L.busy = false;
}

// One scheduling pass: retire finished lanes, then admit waiting requests.
static void schedule(pjac_server* s) {
    for (auto& L : s->lanes) {
        if (!L.busy) continue;
        cudaError_t e = cudaEventQuery(L.done);
        if (e == cudaSuccess) finish_lane(s, L, PJAC_OK);
        else if (e != cudaErrorNotReady) { cudaGetLastError(); finish_lane(s, L, PJAC_ECUDA); }
    }
    const int cluster = s->o.solver.cluster_size;
    auto sms_of = [cluster](int n) { return cluster > 0 ? cluster : jacobi_auto_cluster(n); };
    while (Lane* lp = serve_admit(s->q, s->lanes, sms_of)) {
        Lane& L = *lp;
        s->inflight += (int64_t)L.reqs.size();
        s->peak_inflight = std::max(s->peak_inflight, s->inflight);
        s->peak_hbm = std::max(s->peak_hbm, s->q.in_use);
        L.busy = true;
        int r = launch_lane(s, L);
        if (r != PJAC_OK) finish_lane(s, L, r);
    }
}

extern "C" int pjac_serve_submit(pjac_server* s, const double* A, int n, int lda, pjac_pivot pivot, double tol,
                                 double* W, double* V, int ldv, uint64_t* ticket) {
    if (!s || !A || !W || !ticket) return set_err(PJAC_EINVAL, "NULL argument");
    if (n < 2 || n > PJAC_MAX_N) return set_err(PJAC_EINVAL, "serve: n = %d outside [2, %d]", n, PJAC_MAX_N);
    if (lda < n || (V && ldv < n)) return set_err(PJAC_EINVAL, "serve: leading dimension < n");
    if (pivot < PJAC_PIVOT_GAP || pivot > PJAC_PIVOT_RANDOM) return set_err(PJAC_EINVAL, "bad pivot");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->q.waiting() >= s->o.max_queue)
        return set_err(PJAC_EAGAIN, "serve: queue full");
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < n; ++r) {
            double v = A[r + (size_t)c * lda];
            if (!std::isfinite(v) || v != A[c + (size_t)r * lda])
                return set_err(PJAC_EINVAL, "serve: input has NaN/Inf or is not symmetric");
        }
    Request* q = new Request();
    q->ticket = s->next_ticket++;
    q->n = n;
    q->pivot = pivot;
    q->tol = tol;
    q->a.resize((size_t)n * n);
    for (int c = 0; c < n; ++c) memcpy(q->a.data() + (size_t)c * n, A + (size_t)c * lda, (size_t)n * 8);
    q->w_out = W;
    q->v_out = V;
    q->ldv = ldv;
    q->t_submit = now_ms();
    q->footprint = request_footprint(n);
    if (s->first_submit < 0) s->first_submit = q->t_submit;
    s->q.push(q);
    s->all[q->ticket] = q;
    *ticket = q->ticket;
    schedule(s);
    return PJAC_OK;
}

extern "C" int pjac_serve_poll(pjac_server* s, uint64_t ticket, pjac_info* info) {
    if (!s) return set_err(PJAC_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    schedule(s);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_err(PJAC_EINVAL, "serve: unknown or already collected ticket");
    Request* q = it->second;
    if (q->status == PJAC_PENDING) return PJAC_PENDING;
    if (info) *info = q->info;
    int st = q->status;
    s->all.erase(it);
    delete q;
    return st;
}

extern "C" int pjac_serve_progress(pjac_server* s) {
    if (!s) return set_err(PJAC_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    schedule(s);
    return (int)(s->q.waiting() + s->inflight);
}

extern "C" int pjac_serve_get_stats(pjac_server* s, pjac_serve_stats* st) {
    if (!s || !st) return set_err(PJAC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    std::vector<double> v = s->lat_ms;
    st->completed = (int64_t)v.size();
    st->peak_inflight = s->peak_inflight;
    st->peak_hbm_bytes = s->peak_hbm;
    st->launches = s->launches;
    if (v.empty()) return PJAC_OK;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        double idx = p * (double)(v.size() - 1);
        size_t lo = (size_t)idx;
        size_t hi = std::min(v.size() - 1, lo + 1);
        double f = idx - (double)lo;
        return v[lo] * (1.0 - f) + v[hi] * f;
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_ms = sum / (double)v.size();
    double span = (s->last_done - s->first_submit) / 1000.0;
    st->solves_per_s = span > 0 ? (double)v.size() / span : 0.0;
    return PJAC_OK;
}
