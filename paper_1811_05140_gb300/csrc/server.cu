// Continuous-batching serving loop over the compressed simulator.
//
// A host thread owns every GPU-side object.  Requests (circuits) arrive at
// any time through qsim_server_submit; the loop admits waiting requests
// while the reservations of the resident circuits plus the new circuit's
// stay inside the memory budget (not their 2^(n+4)-byte uncompressed
// size).  A circuit's reservation is the larger of its measured device
// footprint and its growth bound: tables plus two arenas of the codec's
// stream bound (for AALC the ratio threshold's 16 * 2^n / theta bytes).
// Then it runs one tick: the next few sweeps
// of every resident circuit (cut at the circuit's own sweep boundaries, so
// each pass is exactly the one it would run alone) as one batched flush
// (qsim_flush_batch), so circuits that arrived meanwhile join at the next
// tick and their work overlaps on the device with the circuits already
// running.  A circuit whose gates are all applied is read out
// (probabilities of its requested qubits), its memory is released, and its
// latency recorded.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qsim.h"

unsigned long long qs_handle_footprint(qsim_t h);
unsigned long long qs_stream_bound(int n, int c, int codec, double eps, double theta);

namespace {

struct Req {
    unsigned long long id = 0;
    qsim_request r{};
    std::vector<qsim_gate_rec> gates;
    qsim_t h = nullptr;
    size_t next = 0;                    // next gate to queue
    std::vector<size_t> bounds;         // first gate of every sweep, then n_gates
    size_t next_sweep = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int status = QSIM_OK;
    bool done = false;
    std::vector<double> probs;
    unsigned long long stream_bytes = 0, peak_fp = 0;
};

}  // namespace

struct qsim_server {
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> waiting;
    std::vector<Req *> resident;
    std::unordered_map<unsigned long long, Req *> all;
    std::thread th;
    bool stop = false;
    unsigned long long budget = 0;
    int max_resident = 64;
    int sweeps_per_tick = 4;
    int use_graph = 0;
    std::chrono::steady_clock::time_point t0;
    cudaStream_t stream = nullptr;
    int device = 0;
    unsigned long long next_id = 1;
    // statistics
    unsigned long long submitted = 0, completed = 0, failed = 0, ticks = 0, rounds = 0;
    unsigned long long peak_footprint = 0;
    int max_resident_seen = 0;
    double first_submit = -1, last_finish = 0, busy_s = 0;
    std::vector<double> latencies;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void loop();
};

namespace {

int tile_log2_of(const qsim_request &r) {
    return r.tile_log2 ? r.tile_log2 : std::min(std::min(r.block_log2, r.n_qubits), 8);
}

// initial device bytes of a fresh state (tables, norm partials, two arenas)
unsigned long long initial_footprint(const qsim_request &r) {
    int c = tile_log2_of(r);
    unsigned long long ntiles = 1ull << (r.n_qubits - c);
    unsigned long long tile = 32ull + (16ull << c);
    unsigned long long a0 = ntiles * 32ull + tile;
    unsigned long long a1 = std::max<unsigned long long>(a0 + a0 / 4 + (1ull << 20), 1ull << 22);
    a0 = std::max<unsigned long long>(a0, 1ull << 22);
    return ntiles * 32ull + a0 + a1;
}

// growth bound of a circuit: tables and norm partials plus two arenas
// (2 MiB granules, 4 MiB at least) of the codec's stream bound
unsigned long long growth_bound(const qsim_request &r) {
    const int c = tile_log2_of(r);
    const unsigned long long ntiles = 1ull << (r.n_qubits - c);
    const unsigned long long sb = qs_stream_bound(r.n_qubits, c, r.codec, r.rel_err_bound, r.theta);
    const unsigned long long arena = std::max<unsigned long long>((sb + (2ull << 20) - 1) & ~((2ull << 20) - 1),
                                                                  4ull << 20);
    return ntiles * 32ull + 2ull * arena;
}

// bytes a circuit holds or may grow to: the larger of its measured
// footprint (initial before admission) and its growth bound
unsigned long long reservation(const qsim_request &r, qsim_t h) {
    const unsigned long long now = h ? qs_handle_footprint(h) : initial_footprint(r);
    return std::max(now, growth_bound(r));
}

void finish(qsim_server *S, Req *q, int status) {
    q->status = status;
    if (status == QSIM_OK && q->h) {
        size_t nb = (size_t)1 << q->r.n_readout;
        q->probs.assign(nb, 0.0);
        int st = qsim_probabilities(q->h, q->r.readout, q->r.n_readout, q->probs.data());
        unsigned long long sb = 0;
        if (st == QSIM_OK) st = qsim_compressed_bytes(q->h, &sb, nullptr);
        q->stream_bytes = sb;
        q->status = st;
    }
    if (q->h) qsim_destroy(q->h);
    q->h = nullptr;
    q->t_finish = S->now();
    std::lock_guard<std::mutex> lk(S->m);
    q->done = true;
    if (q->status == QSIM_OK) {
        S->completed++;
        S->latencies.push_back(q->t_finish - q->t_submit);
        S->last_finish = q->t_finish;
    } else {
        S->failed++;
    }
    S->cv_done.notify_all();
}

int admit(qsim_server *S, Req *q) {
    const qsim_request &r = q->r;
    int st = qsim_create(&q->h, r.n_qubits, r.block_log2, (qsim_codec)r.codec, r.rel_err_bound);
    if (st != QSIM_OK) return st;
    if ((st = qsim_set_stream(q->h, S->stream)) != QSIM_OK) return st;
    if (r.codec == QSIM_CODEC_AALC && r.theta > 0) {
        const double lad[4] = {1e-5, 1e-4, 1e-3, 1e-2};
        double lv[4];
        int nl = 0;
        for (double e : lad)
            if (e <= r.rel_err_bound * (1 + 1e-12)) lv[nl++] = e;
        if ((st = qsim_set_aalc(q->h, r.theta, lv, nl)) != QSIM_OK) return st;
    }
    if (r.tile_log2 || r.hmax || r.depth) {
        qsim_stats_t d;
        if ((st = qsim_stats(q->h, &d)) != QSIM_OK) return st;
        st = qsim_set_schedule(q->h, r.tile_log2 ? r.tile_log2 : d.tile_log2, r.hmax ? r.hmax : d.hmax,
                               r.depth ? r.depth : d.depth);
        if (st != QSIM_OK) return st;
    }
    if (r.sweep_threads && (st = qsim_set_sweep_threads(q->h, r.sweep_threads)) != QSIM_OK) return st;
    if (r.basis && (st = qsim_reset_basis(q->h, r.basis)) != QSIM_OK) return st;
    // the circuit's own sweep partition: ticks cut only at sweep boundaries,
    // so every pass is the one the circuit would run alone
    qsim_stats_t ss;
    if ((st = qsim_stats(q->h, &ss)) != QSIM_OK) return st;
    const int ng = (int)q->gates.size();
    std::vector<int> nt(ng), tg(2 * (size_t)ng), lo(ng + 1), hh(ng + 1), HH(4 * ((size_t)ng + 1));
    std::vector<double> mats(32 * (size_t)ng);
    for (int i = 0; i < ng; ++i) {
        nt[i] = q->gates[i].n_targets;
        tg[2 * i] = q->gates[i].targets[0];
        tg[2 * i + 1] = q->gates[i].targets[1];
        std::memcpy(&mats[32 * (size_t)i], q->gates[i].matrix, 32 * sizeof(double));
    }
    const int nsw = ng ? qsim_plan_sweeps(r.n_qubits, ss.tile_log2, ss.hmax, ss.depth, ng, nt.data(), tg.data(),
                                          mats.data(), lo.data(), hh.data(), HH.data(), ng + 1)
                       : 0;
    if (nsw < 0) return QSIM_ERR_ARG;
    q->bounds.assign(lo.begin(), lo.begin() + nsw);
    q->bounds.push_back((size_t)ng);
    return QSIM_OK;
}

}  // namespace

void qsim_server::loop() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<Req *> admitted;
        {
            std::unique_lock<std::mutex> lk(m);
            cv_work.wait(lk, [&] { return stop || !waiting.empty() || !resident.empty(); });
            if (stop && waiting.empty() && resident.empty()) return;
            // admission by reservation: every resident circuit's measured
            // footprint or growth bound, whichever is larger, plus the
            // newcomer's; a circuit alone is always admitted
            unsigned long long fp = 0;
            for (Req *q : resident) fp += reservation(q->r, q->h);
            while (!waiting.empty() && (int)(resident.size() + admitted.size()) < max_resident) {
                Req *q = waiting.front();
                const unsigned long long need = reservation(q->r, nullptr);
                const bool empty = resident.empty() && admitted.empty();
                if (!empty && fp + need > budget) break;
                waiting.pop_front();
                admitted.push_back(q);
                fp += need;
            }
        }
        for (Req *q : admitted) {
            q->t_admit = now();
            int st = admit(this, q);
            if (st != QSIM_OK) { finish(this, q, st); continue; }
            resident.push_back(q);
        }
        if (resident.empty()) continue;
        const double tick0 = now();
        // one tick: the next slice of every resident circuit, batched
        std::vector<qsim_t> hs;
        for (Req *q : resident) {
            const size_t nsw = q->bounds.size() - 1;
            q->next_sweep = std::min(nsw, q->next_sweep + (size_t)sweeps_per_tick);
            const size_t end = q->bounds[q->next_sweep];
            int st = QSIM_OK;
            for (; q->next < end && st == QSIM_OK; ++q->next) {
                const qsim_gate_rec &g = q->gates[q->next];
                int ctl[64], nc = 0;
                unsigned long long vals = 0;
                for (int b = 0; b < 64; ++b)
                    if ((g.control_mask >> b) & 1ull) {
                        if ((g.control_values >> b) & 1ull) vals |= 1ull << nc;
                        ctl[nc++] = b;
                    }
                st = qsim_apply_gate(q->h, g.matrix, g.targets, g.n_targets, ctl, nc, vals);
            }
            if (st != QSIM_OK) q->status = st;
            hs.push_back(q->h);
        }
        int st = qsim_flush_batch(hs.data(), (int)hs.size(), use_graph);
        ticks++;
        unsigned long long fp = 0;
        std::vector<Req *> keep;
        for (Req *q : resident) {
            if (q->status == QSIM_OK && st != QSIM_OK) {
                // find out which handle failed: a failed handle reports an invalid state
                qsim_stats_t ss;
                if (qsim_flush(q->h) != QSIM_OK || qsim_stats(q->h, &ss) != QSIM_OK) q->status = QSIM_ERR_CUDA;
            }
            const unsigned long long f = q->h ? qs_handle_footprint(q->h) : 0;
            q->peak_fp = std::max(q->peak_fp, f);
            fp += f;
            if (q->status != QSIM_OK || q->next >= q->gates.size()) finish(this, q, q->status);
            else keep.push_back(q);
        }
        resident.swap(keep);
        peak_footprint = std::max(peak_footprint, fp);
        max_resident_seen = std::max<int>(max_resident_seen, (int)hs.size());
        busy_s += now() - tick0;
    }
}

extern "C" {

qsim_status qsim_server_create(qsim_server_t *out, unsigned long long mem_budget_bytes, int max_resident,
                               int sweeps_per_tick, int use_graph) {
    if (!out || max_resident < 1 || sweeps_per_tick < 1 || mem_budget_bytes < (64ull << 20)) return QSIM_ERR_ARG;
    *out = nullptr;
    qsim_server *S = new qsim_server();
    S->budget = mem_budget_bytes;
    S->max_resident = max_resident;
    S->sweeps_per_tick = sweeps_per_tick;
    S->use_graph = use_graph;
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return QSIM_ERR_CUDA;
    }
    S->th = std::thread([S] { S->loop(); });
    *out = S;
    return QSIM_OK;
}

qsim_status qsim_server_submit(qsim_server_t S, const qsim_request *req, unsigned long long *ticket) {
    if (!S || !req || !ticket || req->n_gates < 0 || (req->n_gates && !req->gates) || req->n_readout < 0 ||
        req->n_readout > 16 || req->n_qubits < 1 || req->n_qubits > 40)
        return QSIM_ERR_ARG;
    Req *q = new Req();
    q->r = *req;
    q->r.gates = nullptr;
    q->gates.assign(req->gates, req->gates + req->n_gates);
    std::lock_guard<std::mutex> lk(S->m);
    if (S->stop) { delete q; return QSIM_ERR_STATE_INVALID; }
    q->id = S->next_id++;
    q->t_submit = S->now();
    if (S->first_submit < 0) S->first_submit = q->t_submit;
    S->all[q->id] = q;
    S->waiting.push_back(q);
    S->submitted++;
    *ticket = q->id;
    S->cv_work.notify_one();
    return QSIM_OK;
}

qsim_status qsim_server_result(qsim_server_t S, unsigned long long ticket, qsim_ticket_info *info,
                               double *probs) {
    if (!S || !info) return QSIM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QSIM_ERR_ARG;
    Req *q = it->second;
    info->done = q->done;
    info->status = q->status;
    info->submit_s = q->t_submit;
    info->admit_s = q->t_admit;
    info->finish_s = q->t_finish;
    info->stream_bytes = q->stream_bytes;
    info->peak_footprint = q->peak_fp;
    if (q->done && probs && !q->probs.empty()) std::memcpy(probs, q->probs.data(), q->probs.size() * sizeof(double));
    return QSIM_OK;
}

qsim_status qsim_server_wait(qsim_server_t S, unsigned long long ticket, double timeout_s) {
    if (!S) return QSIM_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->m);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QSIM_ERR_ARG;
    Req *q = it->second;
    bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return q->done; });
    return ok ? QSIM_OK : QSIM_ERR_TIMEOUT;
}

qsim_status qsim_server_drain(qsim_server_t S, double timeout_s) {
    if (!S) return QSIM_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->m);
    bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                  [&] { return S->completed + S->failed == S->submitted; });
    return ok ? QSIM_OK : QSIM_ERR_TIMEOUT;
}

qsim_status qsim_server_stats(qsim_server_t S, qsim_server_stats_t *out) {
    if (!S || !out) return QSIM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->m);
    qsim_server_stats_t o{};
    o.submitted = S->submitted;
    o.completed = S->completed;
    o.failed = S->failed;
    o.ticks = S->ticks;
    o.peak_footprint = S->peak_footprint;
    o.budget = S->budget;
    o.busy_s = S->busy_s;
    o.max_resident_seen = S->max_resident_seen;
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
        auto pct = [&](double p) {
            size_t i = (size_t)(p * (double)(l.size() - 1) + 0.5);
            return l[std::min(i, l.size() - 1)];
        };
        o.p50_latency_s = pct(0.50);
        o.p99_latency_s = pct(0.99);
        double s = 0;
        for (double x : l) s += x;
        o.mean_latency_s = s / (double)l.size();
        const double span = S->last_finish - S->first_submit;
        o.throughput_cps = span > 0 ? (double)S->completed / span : 0.0;
    }
    *out = o;
    return QSIM_OK;
}

qsim_status qsim_server_destroy(qsim_server_t S) {
    if (!S) return QSIM_OK;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->all) {
        if (kv.second->h) qsim_destroy(kv.second->h);
        delete kv.second;
    }
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    return QSIM_OK;
}

}  // extern "C"
