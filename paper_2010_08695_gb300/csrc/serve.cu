// Serving engine: tip decompositions submitted as they arrive, admitted by
// device memory, run concurrently on worker streams, with small requests
// packed together into one disjoint-union decomposition (continuous
// batching). Host C++ only; every step of the method runs in the kernels of
// the other translation units.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace receipt {
void decompose_batch_impl(receipt_graph *const *gs, const receipt_side *sides, int32_t n,
                          uint64_t *const *d_tips, const receipt_options *opt, cudaStream_t s);
}

using namespace receipt;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    const int32_t *h_eu = nullptr;
    const int32_t *h_ev = nullptr;
    int64_t m = 0;
    int32_t nu = 0, nv = 0;
    int side = 0;
    uint64_t *h_tip = nullptr;
    size_t est = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    bool done = false;
    receipt_status status = RECEIPT_OK;
    std::string err;
};

// Device bytes a request may hold while it runs (graph, build and
// decomposition temporaries), an upper estimate. It includes what a recount
// of Sec. 4.1 allocates when the rule picks one (the remaining subgraph's
// lists, offsets and counts, the counting pass's temporaries and its
// global-tier counters per CTA, a copy of the other side's lists: the sizes
// the decomposition itself checks before recounting) and the fine-grained
// step's global counters of split heavy levels (32 members x the side).
size_t estimate_bytes(int64_t m, int32_t nu, int32_t nv, int side, int sms) {
    const int64_t ns = side ? nv : nu;
    size_t b = (size_t)160 * (size_t)m + (size_t)400 * (size_t)(nu + nv) + ((size_t)32 << 20);
    if (m >= 65535) b += (size_t)8 * 80 * (size_t)ns;  // hub slots of the global tier
    const size_t n_max = (size_t)std::max(nu, nv);
    b += (size_t)40 * (size_t)m + (size_t)48 * (size_t)(nu + nv) + (size_t)8 * (size_t)sms * n_max +
         ((size_t)64 << 20);
    b += (size_t)8 * 32 * (size_t)ns;
    return b;
}

}  // namespace

struct receipt_server {
    receipt_server_config cfg{};
    int device = 0;
    int sms = 1;  // the device's SM count (per-CTA counters of the estimate)
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<int64_t, Request *> reqs;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_id = 1;
    size_t inflight_bytes = 0, peak_bytes = 0;
    int inflight = 0, peak_inflight = 0;
    int64_t submitted = 0, completed = 0, failed = 0, batches = 0, packed = 0;
    double t_first = -1, t_last = -1;
    std::vector<double> lat;

    void worker_loop(int w);
    bool take(std::vector<Request *> &out);
    void run(std::vector<Request *> &batch, cudaStream_t s);
};

// Admission (called with mu held): the oldest pending request is admitted
// if its estimate fits the free budget (or nothing else is running); when it
// is small, later small requests that also fit join it in one batch.
bool receipt_server::take(std::vector<Request *> &out) {
    if (pending.empty()) return false;
    Request *h = pending.front();
    if (inflight > 0 && inflight_bytes + h->est > budget) return false;
    out.push_back(h);
    pending.pop_front();
    size_t bytes = h->est;
    if (h->m <= cfg.batch_max_edges) {
        int64_t edges = h->m;
        for (auto it = pending.begin();
             it != pending.end() && (int)out.size() < cfg.batch_max_graphs;) {
            Request *r = *it;
            if (r->m <= cfg.batch_max_edges && edges + r->m <= (int64_t)cfg.batch_max_edges * 4 &&
                inflight_bytes + bytes + r->est <= budget) {
                out.push_back(r);
                bytes += r->est;
                edges += r->m;
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
    }
    inflight_bytes += bytes;
    inflight++;
    peak_bytes = std::max(peak_bytes, inflight_bytes);
    peak_inflight = std::max(peak_inflight, inflight);
    return true;
}

void receipt_server::run(std::vector<Request *> &batch, cudaStream_t s) {
    const double t0 = now_ms();
    for (Request *r : batch) r->t_start = t0;
    receipt_options opt;
    receipt_options_default(&opt);
    opt.P = cfg.P > 0 ? cfg.P : 150;
    std::vector<receipt_graph *> gs;
    std::vector<DevBuf<unsigned long long>> tips;
    receipt_status st = RECEIPT_OK;
    std::string err;
    try {
        for (Request *r : batch) {
            DevBuf<int32_t> eu(r->m, s), ev(r->m, s);
            if (r->m > 0) {
                RC_CUDA(cudaMemcpyAsync(eu.get(), r->h_eu, 4 * r->m, cudaMemcpyHostToDevice, s));
                RC_CUDA(cudaMemcpyAsync(ev.get(), r->h_ev, 4 * r->m, cudaMemcpyHostToDevice, s));
            }
            gs.push_back(build_graph(eu.get(), ev.get(), r->m, r->nu, r->nv, 1, s));
            tips.emplace_back((size_t)(r->side ? r->nv : r->nu), s);
        }
        if (batch.size() == 1) {
            tip_decompose_impl(gs[0], batch[0]->side, (uint64_t *)tips[0].get(), &opt, s);
        } else {
            std::vector<receipt_side> sides;
            std::vector<uint64_t *> outs;
            for (size_t i = 0; i < batch.size(); i++) {
                sides.push_back((receipt_side)batch[i]->side);
                outs.push_back((uint64_t *)tips[i].get());
            }
            decompose_batch_impl(gs.data(), sides.data(), (int32_t)gs.size(), outs.data(), &opt, s);
        }
        for (size_t i = 0; i < batch.size(); i++) {
            Request *r = batch[i];
            const int32_t n = r->side ? r->nv : r->nu;
            if (n > 0)
                RC_CUDA(cudaMemcpyAsync(r->h_tip, tips[i].get(), 8 * (size_t)n,
                                        cudaMemcpyDeviceToHost, s));
        }
        RC_CUDA(cudaStreamSynchronize(s));
    } catch (const ReceiptError &e) {
        st = e.status;
        err = e.msg;
        cudaStreamSynchronize(s);
    } catch (const std::exception &e) {
        st = RECEIPT_ERR_INTERNAL;
        err = e.what();
        cudaStreamSynchronize(s);
    }
    for (receipt_graph *g : gs) destroy_graph(g);
    tips.clear();
    const double t1 = now_ms();
    std::lock_guard<std::mutex> lk(mu);
    size_t bytes = 0;
    for (Request *r : batch) {
        r->t_done = t1;
        r->status = st;
        r->err = err;
        r->done = true;
        bytes += r->est;
        if (st == RECEIPT_OK) {
            completed++;
            lat.push_back(r->t_done - r->t_submit);
        } else {
            failed++;
        }
    }
    if (batch.size() > 1) {
        batches++;
        packed += (int64_t)batch.size();
    }
    t_last = std::max(t_last, t1);
    inflight_bytes -= bytes;
    inflight--;
    cv_done.notify_all();
    cv_work.notify_all();
}

void receipt_server::worker_loop(int w) {
    cudaSetDevice(device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || take(batch); });
            if (batch.empty()) break;  // stop with nothing admitted
        }
        run(batch, s);
    }
    cudaStreamDestroy(s);
    (void)w;
}

extern "C" {

void receipt_server_config_default(receipt_server_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->max_inflight = 4;
    c->P = 150;
    c->batch_max_edges = 200000;
    c->batch_max_graphs = 64;
}

receipt_status receipt_server_create(const receipt_server_config *cfg, receipt_server **out) {
    try {
        if (!out) throw ReceiptError{RECEIPT_ERR_INVALID, "null output handle"};
        *out = nullptr;
        receipt_server *sv = new receipt_server();
        receipt_server_config_default(&sv->cfg);
        if (cfg) {
            if (cfg->max_inflight > 0) sv->cfg.max_inflight = cfg->max_inflight;
            if (cfg->mem_budget_bytes > 0) sv->cfg.mem_budget_bytes = cfg->mem_budget_bytes;
            if (cfg->P > 0) sv->cfg.P = cfg->P;
            if (cfg->batch_max_edges >= 0) sv->cfg.batch_max_edges = cfg->batch_max_edges;
            if (cfg->batch_max_graphs > 0) sv->cfg.batch_max_graphs = cfg->batch_max_graphs;
        }
        if (cudaGetDevice(&sv->device) != cudaSuccess) {
            cudaGetLastError();
            delete sv;
            throw ReceiptError{RECEIPT_ERR_CUDA, "no CUDA device"};
        }
        if (cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, sv->device) !=
            cudaSuccess) {
            cudaGetLastError();
            delete sv;
            throw ReceiptError{RECEIPT_ERR_CUDA, "cudaDeviceGetAttribute failed"};
        }
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete sv;
            throw ReceiptError{RECEIPT_ERR_CUDA, "cudaMemGetInfo failed"};
        }
        sv->budget = sv->cfg.mem_budget_bytes > 0 ? (size_t)sv->cfg.mem_budget_bytes
                                                  : (size_t)(0.8 * (double)fr);
        for (int w = 0; w < sv->cfg.max_inflight; w++)
            sv->workers.emplace_back([sv, w] { sv->worker_loop(w); });
        *out = sv;
        set_last_error("");
        return RECEIPT_OK;
    } catch (const ReceiptError &e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return RECEIPT_ERR_INTERNAL;
    }
}

receipt_status receipt_server_submit(receipt_server *sv, const int32_t *h_eu, const int32_t *h_ev,
                                     int64_t m, int32_t nu, int32_t nv, receipt_side side,
                                     uint64_t *h_tip, int64_t *request_id) {
    if (!sv || (m > 0 && (!h_eu || !h_ev)) || m < 0 || nu < 0 || nv < 0 ||
        (side != 0 && side != 1) || ((side ? nv : nu) > 0 && !h_tip)) {
        set_last_error("invalid request");
        return RECEIPT_ERR_INVALID;
    }
    Request *r = new Request();
    r->h_eu = h_eu;
    r->h_ev = h_ev;
    r->m = m;
    r->nu = nu;
    r->nv = nv;
    r->side = (int)side;
    r->h_tip = h_tip;
    r->est = estimate_bytes(m, nu, nv, (int)side, sv->sms);
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            set_last_error("server is shutting down");
            return RECEIPT_ERR_BUSY;
        }
        r->id = sv->next_id++;
        sv->reqs[r->id] = r;
        sv->pending.push_back(r);
        sv->submitted++;
        if (sv->t_first < 0) sv->t_first = r->t_submit;
    }
    sv->cv_work.notify_one();
    if (request_id) *request_id = r->id;
    set_last_error("");
    return RECEIPT_OK;
}

receipt_status receipt_server_wait(receipt_server *sv, int64_t request_id, double timeout_s,
                                   int32_t *request_status, double *latency_ms) {
    if (!sv) {
        set_last_error("null server");
        return RECEIPT_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(request_id);
    if (it == sv->reqs.end()) {
        set_last_error("unknown request id");
        return RECEIPT_ERR_INVALID;
    }
    Request *r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s > 0) {
        if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
            set_last_error("request still running");
            return RECEIPT_ERR_TIMEOUT;
        }
    } else {
        sv->cv_done.wait(lk, pred);
    }
    if (request_status) *request_status = (int32_t)r->status;
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    std::string err = r->err;
    sv->reqs.erase(it);
    delete r;
    set_last_error(err);
    return RECEIPT_OK;
}

receipt_status receipt_server_get_stats(receipt_server *sv, receipt_server_stats *out) {
    if (!sv || !out) {
        set_last_error("null argument");
        return RECEIPT_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->batches = sv->batches;
    out->packed_requests = sv->packed;
    out->peak_inflight = sv->peak_inflight;
    out->peak_inflight_bytes = (int64_t)sv->peak_bytes;
    out->budget_bytes = (int64_t)sv->budget;
    std::vector<double> l = sv->lat;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double p) {
            size_t i = (size_t)std::min<double>((double)l.size() - 1, p * (double)(l.size() - 1) + 0.5);
            return l[i];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = l.back();
        double s = 0;
        for (double v : l) s += v;
        out->mean_ms = s / (double)l.size();
        const double span = sv->t_last - sv->t_first;
        out->graphs_per_s = span > 0 ? 1e3 * (double)sv->completed / span : 0.0;
    }
    set_last_error("");
    return RECEIPT_OK;
}

receipt_status receipt_server_destroy(receipt_server *sv) {
    if (!sv) return RECEIPT_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers)
        if (t.joinable()) t.join();
    for (auto &kv : sv->reqs) delete kv.second;
    for (Request *r : sv->pending) (void)r;  // owned by reqs
    delete sv;
    set_last_error("");
    return RECEIPT_OK;
}

}  // extern "C"
