// tune.cu -- the autotuners: a timed solve (or batch) per candidate, the fastest kept.
//  * di_autotune: single solves -- threshold schedule beta, node choice, push grid and
//    direction, then the out-degree class cutoffs;
//  * di_autotune_batch: batched personalized queries of one row width -- class cutoffs,
//    beta, the dense-sweep share that turns the next sweep into a pull, the grid of the
//    batched push and pull, and the row width.
//
// Every candidate is a complete solve to the caller's target, so every result is
// valid (any sequence of diffusions converges to the same X, Section 2.2); the
// candidates only differ in how many sweeps and elementary steps they take and in
// how well the kernels fill the GPU.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "internal.h"

namespace diter {
namespace {

// launch dimensions are part of the captured loops: drop them when the push grid changes
void drop_sweep_graphs(di_graph *g) {
    for (int k = 0; k < kSweepSlots; ++k) {
        if (k == 2) continue;  // the power iteration does not use the push
        if (g->exec[k]) cudaGraphExecDestroy(g->exec[k]);
        if (g->graph[k]) cudaGraphDestroy(g->graph[k]);
        g->exec[k] = nullptr;
        g->graph[k] = nullptr;
    }
    if (g->bp) {
        for (int k = 0; k < kWidths; ++k) {
            if (g->bp->exec[k]) cudaGraphExecDestroy(g->bp->exec[k]);
            if (g->bp->graph[k]) cudaGraphDestroy(g->bp->graph[k]);
            g->bp->exec[k] = nullptr;
            g->bp->graph[k] = nullptr;
        }
    }
}

// a batch width's captured loop holds its grid and dense-sweep share: drop it when they change
void drop_batch_loop(di_graph *g, int slot) {
    if (!g->bp) return;
    if (g->bp->exec[slot]) cudaGraphExecDestroy(g->bp->exec[slot]);
    if (g->bp->graph[slot]) cudaGraphDestroy(g->bp->graph[slot]);
    g->bp->exec[slot] = nullptr;
    g->bp->graph[slot] = nullptr;
}

// the class cutoffs the tuners try; the first is the creation default
constexpr int kCutPairs[][2] = {{kOutCut1, kOutCut2}, {4, 1024}, {8, 256}, {8, 4096}, {4, 256}};

}  // namespace
}  // namespace diter

using namespace diter;

extern "C" di_status di_autotune(di_graph *g, const di_solve_opts *base, di_tune_result *best, di_tune_result *tried,
                                 int32_t cap, int32_t *ntried) {
    if (!g) return set_error(DI_EINVAL, "graph is NULL");
    if (g->untrusted) return set_error(DI_ETIMEOUT, "an earlier sweep scan timed out on this graph: free it");
    if (!base || !best) return set_error(DI_EINVAL, "NULL argument");
    if (!(base->tol > 0.0)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    if (base->prec != DI_FP64 && base->prec != DI_FP32_MIXED)
        return set_error(DI_EINVAL, "prec must be DI_FP64 or DI_FP32_MIXED");
    if (cap > 0 && !tried) return set_error(DI_EINVAL, "tried is NULL");
    const double betas[] = {0.125, 0.25, 0.5, 1.0, 2.0};
    const int grids[] = {2, 4, 8};
    const int selects[] = {DI_SELECT_REF, DI_SELECT_OP, DI_SELECT_OP2};
    const int directions[] = {0, 1};
    const int saved = g->push_per_sm;
    di_tune_result top = {};
    top.ms = -1.0;
    int count = 0;
    for (int pg : grids) {
        if (g->push_per_sm != pg) {
            if (cudaStreamSynchronize(g->stream) != cudaSuccess) return cuda_fail(cudaGetLastError(), "sync");
            drop_sweep_graphs(g);
            g->push_per_sm = pg;
        }
        for (int sel : selects) {
            for (int dir : directions) {
            for (double b : betas) {
                di_solve_opts o = *base;
                o.beta = b;
                o.select = sel;
                o.direction = dir;
                o.trace = 0;
                o.profile = 0;
                o.normalize = 0;
                di_stats st;
                memset(&st, 0, sizeof(st));
                // one run to capture the loop, one timed
                di_status r = run_solve(g, o, nullptr, nullptr, 0, 1.0, nullptr, false, &st);
                if (r == DI_OK) r = run_solve(g, o, nullptr, nullptr, 0, 1.0, nullptr, false, &st);
                if (r != DI_OK && r != DI_ENOTCONVERGED) {
                    g->push_per_sm = saved;
                    drop_sweep_graphs(g);
                    return r;
                }
                di_tune_result t = {};
                t.beta = b;
                t.select = sel;
                t.push_ctas_per_sm = pg;
                t.ms = r == DI_OK ? st.seconds * 1e3 : -1.0;  // a candidate stopped by a limit never wins
                t.edges_pushed = st.edges_pushed;
                t.sweeps = st.sweeps;
                t.direction = dir;
                t.cut1 = g->cut1;
                t.cut2 = g->cut2;
                if (count < cap) tried[count] = t;
                ++count;
                if (t.ms >= 0.0 && (top.ms < 0.0 || t.ms < top.ms)) top = t;
            }
            }
        }
    }
    if (top.ms < 0.0) {
        if (ntried) *ntried = count;
        g->push_per_sm = saved;
        drop_sweep_graphs(g);
        return set_error(DI_ENOTCONVERGED, "no candidate met the target within the limits");
    }
    if (g->push_per_sm != top.push_ctas_per_sm) {
        cudaStreamSynchronize(g->stream);
        drop_sweep_graphs(g);
        g->push_per_sm = top.push_ctas_per_sm;
    }
    // the out-degree class cutoffs, with the fastest of the settings above (the classes are
    // read by the kernels at run time: the captured loops stay valid)
    const int c1_0 = g->cut1, c2_0 = g->cut2;
    for (const auto &cp : kCutPairs) {
        if (cp[0] == top.cut1 && cp[1] == top.cut2) continue;
        di_status r = set_out_classes(g, cp[0], cp[1]);
        if (r != DI_OK) return r;
        di_solve_opts o = *base;
        o.beta = top.beta;
        o.select = top.select;
        o.direction = top.direction;
        o.trace = 0;
        o.profile = 0;
        o.normalize = 0;
        di_stats st;
        memset(&st, 0, sizeof(st));
        r = run_solve(g, o, nullptr, nullptr, 0, 1.0, nullptr, false, &st);
        if (r == DI_OK) r = run_solve(g, o, nullptr, nullptr, 0, 1.0, nullptr, false, &st);
        if (r != DI_OK && r != DI_ENOTCONVERGED) {
            set_out_classes(g, c1_0, c2_0);
            return r;
        }
        di_tune_result t = top;
        t.ms = r == DI_OK ? st.seconds * 1e3 : -1.0;
        t.edges_pushed = st.edges_pushed;
        t.sweeps = st.sweeps;
        t.cut1 = cp[0];
        t.cut2 = cp[1];
        if (count < cap) tried[count] = t;
        ++count;
        if (t.ms >= 0.0 && t.ms < top.ms) top = t;
    }
    if (ntried) *ntried = count;
    if (g->cut1 != top.cut1 || g->cut2 != top.cut2) {
        di_status r = set_out_classes(g, top.cut1, top.cut2);
        if (r != DI_OK) return r;
    }
    *best = top;
    return DI_OK;
}

extern "C" di_status di_autotune_batch(di_graph *g, int32_t k, const int32_t *seed_ptr, const int32_t *seeds,
                                       const double *w, double tol, di_batch_tune_result *best,
                                       di_batch_tune_result *tried, int32_t cap, int32_t *ntried) {
    if (!g) return set_error(DI_EINVAL, "graph is NULL");
    if (g->untrusted) return set_error(DI_ETIMEOUT, "an earlier sweep scan timed out on this graph: free it");
    if (!best) return set_error(DI_EINVAL, "best is NULL");
    if (cap > 0 && !tried) return set_error(DI_EINVAL, "tried is NULL");
    std::vector<int32_t> hp, hs;
    std::vector<double> hw;
    if (di_status r = batch_args(g, k, seed_ptr, seeds, w, tol, hp, hs, hw); r != DI_OK) return r;
    const int nat = lane_slot(k);
    std::vector<di_stats> stq((size_t)k);
    int count = 0;
    // the current settings of the natural width; the width setting selects the slot that runs
    BatchTune cur = g->btune[nat];
    cur.exec_slot = -1;
    int slot = nat;
    di_batch_tune_result top = {};
    top.ms = -1.0;
    // one timed batch with settings `bt` on width `sl` (the first run captures the loop)
    auto trial = [&](const BatchTune &bt, int sl, di_batch_tune_result &t) -> di_status {
        const BatchTune keep_nat = g->btune[nat], keep_sl = g->btune[sl];
        BatchTune run = bt;
        run.exec_slot = -1;
        if (g->btune[sl].pull_share != run.pull_share || g->btune[sl].push_per_sm != run.push_per_sm) {
            cudaStreamSynchronize(g->stream);
            drop_batch_loop(g, sl);
        }
        g->btune[sl] = run;
        g->btune[nat].exec_slot = sl == nat ? -1 : sl;
        di_stats all;
        memset(&all, 0, sizeof(all));
        di_status r = run_query_batch(g, k, hp.data(), hs.data(), w ? hw.data() : nullptr, tol, bt.beta, 1000000,
                                      nullptr, false, stq.data(), &all, nullptr);
        if (r == DI_OK) r = run_query_batch(g, k, hp.data(), hs.data(), w ? hw.data() : nullptr, tol, bt.beta,
                                            1000000, nullptr, false, stq.data(), &all, nullptr);
        // put the slots back as they were: the caller decides what stays
        if (keep_sl.pull_share != run.pull_share || keep_sl.push_per_sm != run.push_per_sm) {
            cudaStreamSynchronize(g->stream);
            drop_batch_loop(g, sl);
        }
        g->btune[sl] = keep_sl;
        if (sl != nat) g->btune[nat] = keep_nat;
        if (r != DI_OK && r != DI_ENOTCONVERGED) return r;
        t = {};
        t.beta = bt.beta;
        t.ms = r == DI_OK ? all.seconds * 1e3 : -1.0;
        t.max_bound = all.bound;
        t.edges_pushed = all.edges_pushed;
        t.sweeps = all.sweeps;
        t.lanes = slot_width(sl);
        t.pull_share = bt.pull_share;
        t.push_ctas_per_sm = bt.push_per_sm;
        t.cut1 = g->cut1;
        t.cut2 = g->cut2;
        if (count < cap) tried[count] = t;
        ++count;
        return DI_OK;
    };
    auto better = [&](const di_batch_tune_result &t) { return t.ms >= 0.0 && (top.ms < 0.0 || t.ms < top.ms); };
    const int c1_0 = g->cut1, c2_0 = g->cut2;
    di_batch_tune_result t;
    // 1. class cutoffs
    int bc1 = c1_0, bc2 = c2_0;
    for (const auto &cp : kCutPairs) {
        if (count > 0 && cp[0] == bc1 && cp[1] == bc2) continue;
        di_status r = set_out_classes(g, cp[0], cp[1]);
        if (r == DI_OK) r = trial(cur, slot, t);
        if (r != DI_OK) {
            set_out_classes(g, c1_0, c2_0);
            return r;
        }
        if (better(t)) {
            top = t;
            bc1 = cp[0];
            bc2 = cp[1];
        }
    }
    if (g->cut1 != bc1 || g->cut2 != bc2) {
        if (di_status r = set_out_classes(g, bc1, bc2); r != DI_OK) return r;
    }
    // 2. beta, 3. dense-sweep share, 4. grid: each with the best so far
    const double betas[] = {0.25, 0.5, 1.0};
    const int shares[] = {2, 4, 8, 16};
    const int grids[] = {2, 4, 8};
    for (double b : betas) {
        if (b == cur.beta) continue;
        BatchTune c = cur;
        c.beta = b;
        if (di_status r = trial(c, slot, t); r != DI_OK) return r;
        if (better(t)) { top = t; cur = c; }
    }
    for (int sh : shares) {
        if (sh == cur.pull_share) continue;
        BatchTune c = cur;
        c.pull_share = sh;
        if (di_status r = trial(c, slot, t); r != DI_OK) return r;
        if (better(t)) { top = t; cur = c; }
    }
    for (int gr : grids) {
        if (gr == cur.push_per_sm) continue;
        BatchTune c = cur;
        c.push_per_sm = gr;
        if (di_status r = trial(c, slot, t); r != DI_OK) return r;
        if (better(t)) { top = t; cur = c; }
    }
    // 5. the next wider row
    if (nat + 1 < kWidths) {
        if (di_status r = trial(cur, nat + 1, t); r != DI_OK) return r;
        if (better(t)) { top = t; slot = nat + 1; }
    }
    if (ntried) *ntried = count;
    if (top.ms < 0.0) return set_error(DI_ENOTCONVERGED, "no candidate batch met the target within the limits");
    // keep the winner for batches of this width
    cudaStreamSynchronize(g->stream);
    drop_batch_loop(g, slot);
    cur.tuned = 1;
    cur.exec_slot = -1;
    g->btune[slot] = cur;
    g->btune[nat].exec_slot = slot == nat ? -1 : slot;
    if (slot != nat) g->btune[nat].tuned = 1;
    *best = top;
    return DI_OK;
}
