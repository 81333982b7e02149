// tune.cu -- the autotuner: a timed solve per candidate (threshold schedule beta,
// node choice, push grid, direction), the fastest kept.
//
// Every candidate is a complete solve to the caller's target, so every result is
// valid (any sequence of diffusions converges to the same X, Section 2.2); the
// candidates only differ in how many sweeps and elementary steps they take and in
// how well the push fills the GPU.
#include <cuda_runtime.h>

#include <cstring>

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
                if (count < cap) tried[count] = t;
                ++count;
                if (t.ms >= 0.0 && (top.ms < 0.0 || t.ms < top.ms)) top = t;
            }
            }
        }
    }
    if (ntried) *ntried = count;
    if (top.ms < 0.0) {
        g->push_per_sm = saved;
        drop_sweep_graphs(g);
        return set_error(DI_ENOTCONVERGED, "no candidate met the target within the limits");
    }
    if (g->push_per_sm != top.push_ctas_per_sm) {
        cudaStreamSynchronize(g->stream);
        drop_sweep_graphs(g);
        g->push_per_sm = top.push_ctas_per_sm;
    }
    *best = top;
    return DI_OK;
}
