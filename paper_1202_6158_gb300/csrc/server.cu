// server.cu -- continuous batching of personalized queries over several graphs.
//
// Each graph gets a lane pool (BatchPool, batch.cu): K interleaved query lanes and
// its own CUDA stream.  The host loop (di_server_poll) cycles every pool through
//
//   round     k_bround_begin (free / start lanes), the captured sweep loop for at
//             most round_sweeps sweeps or until a lane stops, the exact FP64
//             |F_q|_1 of the lanes that stopped, and a copy of the lane states
//             to page-locked host memory; an event marks its end.
//   retire    lanes whose stop was confirmed: their H columns are written to the
//             callers' buffers in input numbering and the columns cleared.
//   admit     queued queries take the free lanes: F_q = (1-d) V_q on their seeds.
//
// so lanes are refilled while the others keep diffusing.  Diffusions of different
// queries never interact (each lane is its own fluid), and any order of diffusions
// reaches the same limit (Section 2.2), so a query's result does not depend on
// which queries shared its rounds, beyond the two bounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace diter {
namespace {

struct SrvReq {
    long long ticket = 0;
    std::vector<int> seeds;
    std::vector<double> w;   // empty: uniform over the seeds
    double tol = 0.0;
    double *out = nullptr;   // the caller's buffer (NULL: result dropped)
    double *kout = nullptr;  // the address the retire kernel writes, NULL when staged or dropped
    double t_submit = 0.0, t_admit = 0.0;
    bool cancelled = false;  // running lane: cleared, not copied out, at the end of its round
};

struct SrvPool {
    di_graph *g = nullptr;
    BatchPool *bp = nullptr;
    int index = 0;           // position in the server's graph list
    int K = 0, slot = 0;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_round = nullptr, ev_ret = nullptr;
    cudaEvent_t ev_start = nullptr;       // timing: recorded before each round's first command
    di_server_graph_stats stats = {};
    bool running = false;
    int round_width = 0;     // lanes per row of the round in flight
    std::deque<SrvReq> queue;
    std::vector<SrvReq> lane;
    std::vector<char> busy;
    unsigned long long retire_mask = 0, admit_mask = 0;  // applied when the next round opens
    LaneAdmin adm = {};
    std::vector<di_completion> ret_wait;  // copied out, waiting for ev_ret
    // seed staging: page-locked host and device copies of (lane, seed, value) items
    int cap_items = 0;
    int *h_q = nullptr, *h_seeds = nullptr, *d_q = nullptr, *d_seeds = nullptr;
    double *h_val = nullptr, *d_val = nullptr;
    double *stage = nullptr;  // device double[n] for results bound for pageable host memory
};

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

di_status grow_items(SrvPool &p, int need) {
    if (need <= p.cap_items) return DI_OK;
    int cap = std::max(need, std::max(1024, 2 * p.cap_items));
    if (p.h_q) {
        DI_CUDA(cudaStreamSynchronize(p.s));
        cudaFreeHost(p.h_q);
        cudaFreeHost(p.h_seeds);
        cudaFreeHost(p.h_val);
        cudaFree(p.d_q);
        cudaFree(p.d_seeds);
        cudaFree(p.d_val);
        p.h_q = p.h_seeds = p.d_q = p.d_seeds = nullptr;
        p.h_val = p.d_val = nullptr;
    }
    DI_CUDA(cudaMallocHost(&p.h_q, sizeof(int) * cap));
    DI_CUDA(cudaMallocHost(&p.h_seeds, sizeof(int) * cap));
    DI_CUDA(cudaMallocHost(&p.h_val, sizeof(double) * cap));
    DI_CUDA(cudaMalloc(&p.d_q, sizeof(int) * cap));
    DI_CUDA(cudaMalloc(&p.d_seeds, sizeof(int) * cap));
    DI_CUDA(cudaMalloc(&p.d_val, sizeof(double) * cap));
    p.cap_items = cap;
    return DI_OK;
}

void free_pool(SrvPool *p) {
    if (!p) return;
    if (p->s) cudaStreamSynchronize(p->s);
    if (p->bp) pool_free(p->bp, p->s);
    if (p->h_q) cudaFreeHost(p->h_q);
    if (p->h_seeds) cudaFreeHost(p->h_seeds);
    if (p->h_val) cudaFreeHost(p->h_val);
    if (p->d_q) cudaFree(p->d_q);
    if (p->d_seeds) cudaFree(p->d_seeds);
    if (p->d_val) cudaFree(p->d_val);
    if (p->stage) cudaFree(p->stage);
    if (p->ev_round) cudaEventDestroy(p->ev_round);
    if (p->ev_ret) cudaEventDestroy(p->ev_ret);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->s) cudaStreamDestroy(p->s);
    cudaGetLastError();
    delete p;
}

}  // namespace
}  // namespace diter

struct di_server {
    std::vector<diter::SrvPool *> pools;
    long long next_ticket = 1;
    int round_sweeps = 16;
    int lane_sweeps = 1 << 20;
    double beta = 0.5;
    std::deque<di_completion> done;
};

namespace diter {
namespace {

void flush_retired(di_server *srv, SrvPool &p, double t) {
    for (di_completion c : p.ret_wait) {
        c.t_done = t;
        srv->done.push_back(c);
    }
    p.ret_wait.clear();
}

// after a round: copy out and clear the lanes whose stop was confirmed
di_status retire_lanes(SrvPool &p) {
    const double omd = 1.0 - p.g->d;
    LaneRetire direct = {};
    std::vector<int> staged;
    for (int q = 0; q < p.K; ++q) {
        if (!p.busy[q]) continue;
        const BatchQ &b = p.bp->h_bq[q];
        const SrvReq &r = p.lane[q];
        if (r.cancelled) {  // cleared only: the caller's buffer is not written, no completion
            direct.lane[direct.count] = q;
            direct.out[direct.count] = nullptr;
            direct.count += 1;
            p.busy[q] = 0;
            p.retire_mask |= 1ull << q;
            continue;
        }
        if (!(b.active && b.done && b.confirmed)) continue;
        di_completion c = {};
        c.ticket = r.ticket;
        c.graph = p.index;
        c.status = b.done == 1 ? DI_OK : DI_ENOTCONVERGED;
        c.bound = b.l1_exact / omd;
        c.sweeps = b.sweeps;
        c.lane = q;
        c.t_submit = r.t_submit;
        c.t_admit = r.t_admit;
        p.ret_wait.push_back(c);
        if (r.out && !r.kout) {
            staged.push_back(q);
        } else {
            direct.lane[direct.count] = q;
            direct.out[direct.count] = r.kout;
            direct.count += 1;
        }
        p.busy[q] = 0;
        p.retire_mask |= 1ull << q;
        p.stats.completed += 1;
    }
    di_status st = pool_retire(p.g, p.bp, p.K, direct, p.s);
    if (st != DI_OK) return st;
    for (int q : staged) {
        LaneRetire one = {};
        one.count = 1;
        one.lane[0] = q;
        one.out[0] = p.stage;
        st = pool_retire(p.g, p.bp, p.K, one, p.s);
        if (st != DI_OK) return st;
        DI_CUDA(cudaMemcpyAsync(p.lane[q].out, p.stage, sizeof(double) * (size_t)p.g->n, cudaMemcpyDeviceToHost,
                                p.s));
    }
    if (!p.ret_wait.empty()) DI_CUDA(cudaEventRecord(p.ev_ret, p.s));
    return DI_OK;
}

// queued queries into free lanes, then the next round if any lane is busy
di_status admit_and_launch(di_server *srv, SrvPool &p, double t) {
    const double omd = 1.0 - p.g->d;
    int nitems = 0;
    std::vector<int> took;
    for (int q = 0; q < p.K && !p.queue.empty(); ++q) {
        if (p.busy[q]) continue;
        took.push_back(q);
        p.lane[q] = std::move(p.queue.front());
        p.queue.pop_front();
        p.lane[q].t_admit = t;
        p.busy[q] = 1;
        nitems += (int)p.lane[q].seeds.size();
    }
    if (!took.empty()) DI_CUDA(cudaEventRecord(p.ev_start, p.s));
    if (nitems) {
        di_status st = grow_items(p, nitems);
        if (st != DI_OK) return st;
        int at = 0;
        for (int q : took) {
            const SrvReq &r = p.lane[q];
            double sum = 0.0;
            for (size_t j = 0; j < r.seeds.size(); ++j) sum += r.w.empty() ? 1.0 : r.w[j];
            for (size_t j = 0; j < r.seeds.size(); ++j, ++at) {
                p.h_q[at] = q;
                p.h_seeds[at] = r.seeds[j];
                p.h_val[at] = omd * (r.w.empty() ? 1.0 : r.w[j]) / sum;
            }
            p.admit_mask |= 1ull << q;
            p.adm.tolR[q] = r.tol * omd;
        }
        DI_CUDA(cudaMemcpyAsync(p.d_q, p.h_q, sizeof(int) * nitems, cudaMemcpyHostToDevice, p.s));
        DI_CUDA(cudaMemcpyAsync(p.d_seeds, p.h_seeds, sizeof(int) * nitems, cudaMemcpyHostToDevice, p.s));
        DI_CUDA(cudaMemcpyAsync(p.d_val, p.h_val, sizeof(double) * nitems, cudaMemcpyHostToDevice, p.s));
        st = pool_seed(p.g, p.bp, p.K, nitems, p.d_q, p.d_seeds, p.d_val, p.s);
        if (st != DI_OK) return st;
    }
    int top = 0;  // lanes 0..top-1 hold every busy lane; the round runs the narrowest loop that covers them
    for (int q = 0; q < p.K; ++q)
        if (p.busy[q]) top = q + 1;
    if (!top) return DI_OK;
    const int wslot = lane_slot(top);
    if (took.empty()) DI_CUDA(cudaEventRecord(p.ev_start, p.s));
    p.stats.admitted += (long long)took.size();
    p.adm.retire = p.retire_mask & ~p.admit_mask;
    p.adm.admit = p.admit_mask;
    di_status st = pool_launch_round(p.g, p.bp, wslot, p.adm, srv->round_sweeps, srv->lane_sweeps, srv->beta, p.s);
    if (st != DI_OK) return st;
    DI_CUDA(cudaEventRecord(p.ev_round, p.s));
    p.round_width = slot_width(wslot);
    p.retire_mask = p.admit_mask = 0;
    p.running = true;
    return DI_OK;
}

// one pass over a pool; *progressed is set when anything changed
di_status step_pool(di_server *srv, SrvPool &p, bool *progressed) {
    if (!p.ret_wait.empty()) {
        cudaError_t e = cudaEventQuery(p.ev_ret);
        if (e == cudaSuccess) {
            flush_retired(srv, p, now_s());
            *progressed = true;
        } else if (e != cudaErrorNotReady) {
            return cuda_fail(e, "cudaEventQuery(retire)");
        }
    }
    if (p.running) {
        cudaError_t e = cudaEventQuery(p.ev_round);
        if (e == cudaErrorNotReady) return DI_OK;
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery(round)");
        p.running = false;
        *progressed = true;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.ev_start, p.ev_round) == cudaSuccess) p.stats.device_ms += ms;
        cudaGetLastError();
        const BatchCtl &c = *p.bp->h_bctl;
        p.stats.rounds += 1;
        p.stats.sweeps += c.round_sweeps;
        p.stats.width_sweeps += (long long)c.round_sweeps * p.round_width;
        p.stats.edges_pushed = c.edges;
        p.stats.sources_pushed = c.srcs;
        // the round ran after the last copy-out on this stream: that copy is complete
        if (!p.ret_wait.empty()) flush_retired(srv, p, now_s());
        di_status st = retire_lanes(p);
        if (st != DI_OK) return st;
    }
    if (!p.running && !p.queue.empty()) *progressed = true;
    return admit_and_launch(srv, p, now_s());
}

}  // namespace
}  // namespace diter

using namespace diter;

extern "C" {

double di_clock(void) { return now_s(); }

di_status di_plan_lanes(const int64_t *lane_bytes, const int64_t *fixed_bytes, int32_t ngraphs, int64_t budget,
                        int32_t *lanes_out) {
    if (!lane_bytes || !fixed_bytes || !lanes_out) return set_error(DI_EINVAL, "NULL argument");
    if (ngraphs < 1) return set_error(DI_EINVAL, "ngraphs must be >= 1");
    for (int i = 0; i < ngraphs; ++i)
        if (lane_bytes[i] < 0 || fixed_bytes[i] < 0) return set_error(DI_EINVAL, "negative byte count");
    std::vector<int> lanes(ngraphs, kLanes);
    auto total = [&]() {
        long double t = 0;
        for (int i = 0; i < ngraphs; ++i) t += (long double)fixed_bytes[i] + (long double)lanes[i] * lane_bytes[i];
        return t;
    };
    if (budget > 0) {
        while (total() > (long double)budget) {
            int pick = -1;
            long double worst = -1;
            for (int i = 0; i < ngraphs; ++i) {
                if (lanes[i] <= 8) continue;
                const long double c = (long double)lanes[i] * lane_bytes[i];
                if (c > worst) {
                    worst = c;
                    pick = i;
                }
            }
            if (pick < 0) return set_error(DI_ENOMEM, "8 lanes per graph do not fit in the memory budget");
            lanes[pick] /= 2;
        }
    }
    for (int i = 0; i < ngraphs; ++i) lanes_out[i] = lanes[i];
    return DI_OK;
}

di_status di_server_create(di_graph *const *graphs, int32_t ngraphs, int64_t mem_budget, int32_t round_sweeps,
                           int32_t lane_sweeps, di_server **out) {
    if (!out) return set_error(DI_EINVAL, "out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs < 1) return set_error(DI_EINVAL, "need at least one graph");
    if (round_sweeps < 1 || round_sweeps > 1024) return set_error(DI_EINVAL, "round_sweeps must be in [1, 1024]");
    if (lane_sweeps < 1) return set_error(DI_EINVAL, "lane_sweeps must be >= 1");
    std::vector<int64_t> lane_b(ngraphs), fixed_b(ngraphs);
    for (int i = 0; i < ngraphs; ++i) {
        if (!graphs[i]) return set_error(DI_EINVAL, "graph " + std::to_string(i) + " is NULL");
        if (graphs[i]->untrusted)
            return set_error(DI_ETIMEOUT, "graph " + std::to_string(i) + " had a sweep scan time out: free it");
        lane_b[i] = pool_bytes(graphs[i], 1) - pool_bytes(graphs[i], 0);
        fixed_b[i] = pool_bytes(graphs[i], 0) + 8LL * graphs[i]->n;
    }
    std::vector<int32_t> lanes(ngraphs);
    di_status st = di_plan_lanes(lane_b.data(), fixed_b.data(), ngraphs, mem_budget, lanes.data());
    if (st != DI_OK) return st;
    di_server *srv = new di_server();
    srv->round_sweeps = round_sweeps;
    srv->lane_sweeps = lane_sweeps;
    auto fail = [&](di_status s) {
        di_server_free(srv);
        return s;
    };
    // smaller graphs get higher stream priority: their short rounds are dispatched
    // ahead of the long rounds of large graphs when both wait for SMs
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaGetLastError();
    std::vector<int> order(ngraphs), rank(ngraphs);
    for (int i = 0; i < ngraphs; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return graphs[a]->n < graphs[b]->n; });
    for (int r = 0; r < ngraphs; ++r) rank[order[r]] = r;
    for (int i = 0; i < ngraphs; ++i) {
        di_graph *g = graphs[i];
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamSynchronize(graph)"));
        SrvPool *p = new SrvPool();
        srv->pools.push_back(p);
        p->g = g;
        p->index = i;
        p->K = lanes[i];
        p->slot = lane_slot(p->K);
        p->lane.resize(p->K);
        p->busy.assign(p->K, 0);
        const int prio = std::max(greatest, least - (ngraphs - 1 - rank[i]));
        e = cudaStreamCreateWithPriority(&p->s, cudaStreamNonBlocking, prio);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreateWithPriority"));
        e = cudaEventCreate(&p->ev_round);
        if (e == cudaSuccess) e = cudaEventCreate(&p->ev_start);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_ret, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate"));
        e = cudaMalloc(&p->stage, sizeof(double) * (size_t)g->n);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(stage)"));
        p->bp = new BatchPool();
        p->bp->stride = p->K;
        if ((st = pool_alloc(g, p->bp, p->K, p->s)) != DI_OK) return fail(st);
        for (int w = 0; w <= p->slot; ++w)
            if ((st = pool_build_loop(g, p->bp, w)) != DI_OK) return fail(st);
        if ((st = pool_reset(g, p->bp, p->K, srv->beta, p->s)) != DI_OK) return fail(st);
        e = cudaStreamSynchronize(p->s);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamSynchronize(pool)"));
    }
    *out = srv;
    return DI_OK;
}

di_status di_server_lanes(const di_server *s, int32_t *lanes_out) {
    if (!s || !lanes_out) return set_error(DI_EINVAL, "NULL argument");
    for (size_t i = 0; i < s->pools.size(); ++i) lanes_out[i] = s->pools[i]->K;
    return DI_OK;
}

di_status di_server_submit(di_server *s, int32_t graph, const int32_t *seeds, const double *w, int32_t nseeds,
                           double tol, double *H_out, int64_t *ticket) {
    if (!s) return set_error(DI_EINVAL, "server is NULL");
    if (graph < 0 || graph >= (int)s->pools.size()) return set_error(DI_EINVAL, "graph index out of range");
    if (nseeds < 1 || !seeds) return set_error(DI_EINVAL, "a query needs at least one seed");
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(DI_EINVAL, "tol must be positive and finite");
    SrvPool &p = *s->pools[graph];
    SrvReq r;
    r.seeds.assign(seeds, seeds + nseeds);
    for (int v : r.seeds)
        if (v < 0 || v >= p.g->n) return set_error(DI_EINVAL, "seed id out of range");
    if (w) {
        r.w.assign(w, w + nseeds);
        double sum = 0.0;
        for (double x : r.w) {
            if (!(x >= 0.0) || !std::isfinite(x)) return set_error(DI_EINVAL, "weights must be finite and >= 0");
            sum += x;
        }
        if (!(sum > 0.0)) return set_error(DI_EINVAL, "weights must not all be zero");
    }
    r.tol = tol;
    r.out = H_out;
    r.kout = H_out ? (double *)kernel_ptr(H_out) : nullptr;
    r.ticket = s->next_ticket++;
    r.t_submit = now_s();
    if (ticket) *ticket = r.ticket;
    p.queue.push_back(std::move(r));
    return DI_OK;
}

di_status di_server_poll(di_server *s, double wait_s, di_completion *out, int32_t cap, int32_t *nout) {
    if (!s) return set_error(DI_EINVAL, "server is NULL");
    if (nout) *nout = 0;
    if (cap > 0 && !out) return set_error(DI_EINVAL, "out is NULL");
    const double t_end = now_s() + std::max(0.0, wait_s);
    for (;;) {
        bool progressed = false;
        for (size_t i = 0; i < s->pools.size(); ++i) {
            di_status st = step_pool(s, *s->pools[i], &progressed);
            if (st != DI_OK) return st;
        }
        bool idle = true;
        for (const SrvPool *p : s->pools) idle &= !p->running && p->queue.empty() && p->ret_wait.empty();
        if (!s->done.empty() || idle || now_s() >= t_end) break;
        if (!progressed) std::this_thread::yield();
    }
    int k = 0;
    while (k < cap && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    if (nout) *nout = k;
    return DI_OK;
}

di_status di_server_cancel(di_server *s, int64_t ticket, int32_t *cancelled) {
    if (!s) return set_error(DI_EINVAL, "server is NULL");
    if (cancelled) *cancelled = 0;
    for (SrvPool *p : s->pools) {
        for (auto it = p->queue.begin(); it != p->queue.end(); ++it) {
            if (it->ticket != ticket) continue;
            p->queue.erase(it);
            p->stats.cancelled += 1;
            if (cancelled) *cancelled = 1;
            return DI_OK;
        }
        for (int q = 0; q < p->K; ++q) {
            if (!p->busy[q] || p->lane[q].ticket != ticket || p->lane[q].cancelled) continue;
            // the lane's round may be in flight: it is cleared when that round ends
            p->lane[q].cancelled = true;
            p->stats.cancelled += 1;
            if (cancelled) *cancelled = 1;
            return DI_OK;
        }
    }
    return DI_OK;
}

di_status di_server_stats(const di_server *s, int32_t graph, di_server_graph_stats *out) {
    if (!s || !out) return set_error(DI_EINVAL, "NULL argument");
    if (graph < 0 || graph >= (int)s->pools.size()) return set_error(DI_EINVAL, "graph index out of range");
    *out = s->pools[graph]->stats;
    out->lanes = s->pools[graph]->K;
    return DI_OK;
}

di_status di_server_pending(const di_server *s, int64_t *queued, int64_t *running) {
    if (!s) return set_error(DI_EINVAL, "server is NULL");
    long long qd = 0, rn = 0;
    for (const SrvPool *p : s->pools) {
        qd += (long long)p->queue.size();
        for (char b : p->busy) rn += b ? 1 : 0;
        rn += (long long)p->ret_wait.size();
    }
    if (queued) *queued = qd;
    if (running) *running = rn;
    return DI_OK;
}

void di_server_free(di_server *s) {
    if (!s) return;
    for (SrvPool *p : s->pools) free_pool(p);
    delete s;
}

}  // extern "C"
