/*
 * diter.h -- C ABI of libditer: D-iteration (fluid diffusion) PageRank on one
 * GB300 GPU (sm_103a).
 *
 * The method is D. Hong, "Optimized on-line computation of PageRank
 * algorithm":
 *   Section 2.1  the problem  X = dPX + (1-d)V  with P_ij the probability of the
 *                move j -> i (column j of P spreads 1/outdeg(j) over the children
 *                of j) and V a normalized personalization vector;
 *   Section 2.2  fluid F_0 = (1-d)V, history H, and ALGO-REF: pick a node, move
 *                its fluid into H, push d*F_i/outdeg_i along every out-link,
 *                decrement the residual R by (1-d)F_i, stop when
 *                R/(1-d) <= target;
 *   Theorem 2    |X - H_n|_1 = |F_n|_1/(1-d)  (an upper bound with dangling
 *                nodes, Section 3.3);
 *   Section 3.3  dangling nodes: their fluid leaves the system (R -= F_i) and P
 *                is never completed;
 *   Section 4.2  threshold sweeps: every node above a threshold diffuses in the
 *                same step and the threshold is lowered progressively.
 *
 * Conventions for every call:
 *   - Node ids are int32 in [0, n).  The graph is a CSR of OUT-links: row i of
 *     (row_ptr, col_idx) lists the children of node i; multi-edges and
 *     self-loops are allowed and each listed edge carries 1/outdeg(i).
 *   - Pointers marked "host or device" may point to either; the library finds
 *     out with cudaPointerGetAttributes.  Inputs are copied at the call; the
 *     caller keeps ownership of every buffer it passes.  Outputs are written
 *     into caller-owned buffers.
 *   - Every call returns a di_status and never aborts; di_last_error() gives a
 *     thread-local message for the last failure.  All work is issued on the
 *     stream given at graph creation; calls that return results synchronize
 *     that stream before returning.
 *   - A di_graph is thread-compatible, not thread-safe: do not use one graph
 *     from two host threads at once.
 */
#ifndef DITER_H
#define DITER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct di_graph di_graph; /* opaque; owns all of its device memory */

typedef enum {
    DI_OK = 0,
    DI_EINVAL = 1,         /* invalid argument or graph (message says which) */
    DI_ENOMEM = 2,         /* device allocation failed */
    DI_ECUDA = 3,          /* a CUDA runtime call failed */
    DI_ENOTCONVERGED = 4,  /* a limit stopped the solve first; outputs are still written */
    DI_ETIMEOUT = 5,       /* a bounded device-side wait gave up */
    DI_EKERNEL = 6         /* a kernel reported an internal error (non-finite residual, ...) */
} di_status;

typedef enum {
    DI_FP64 = 0,        /* fluid, pushes, history and residual all in FP64 */
    DI_FP32_MIXED = 1   /* fluid and pushes in FP32; history and |F|_1 reductions in FP64 */
} di_prec;

typedef struct {
    double bound;          /* |F|_1/(1-d) recomputed exactly at exit: the Theorem 2 bound on |X - H|_1 */
    double l1_F;           /* |F|_1 recomputed at exit (FP64 sum) */
    double R;              /* the tracked residual R of ALGO-REF at exit */
    int64_t edges_pushed;  /* elementary steps (Section 4.2): out-links used by the diffusions */
    int64_t sources_pushed;/* diffusions made (one per selected node per sweep) */
    int32_t sweeps;        /* threshold sweeps (D-iteration) or products (power iteration) */
    int32_t converged;     /* 1 if the stop rule was met */
    double seconds;        /* device time from initialization to the confirmed stop (CUDA events) */
    int64_t kernel_launches; /* kernels this call ran on the GPU (each graph-loop iteration counted) */
} di_stats;

typedef struct {
    double tol;              /* target on |F|_1/(1-d); > 0 */
    double beta;             /* threshold T = beta * R / n before each sweep (default 0.5) */
    int64_t max_edge_pushes; /* stop with DI_ENOTCONVERGED beyond this many elementary steps (<= 0: none) */
    int32_t max_sweeps;      /* stop with DI_ENOTCONVERGED after this many sweeps (<= 0: 1,000,000) */
    int32_t prec;            /* a di_prec value */
    int32_t normalize;       /* 0: raw H (uncompleted P); 1: H/|H|_1 (Section 3.3 renormalization) */
    int32_t trace;           /* 1: record one di_sweep_record per sweep, read with di_get_trace */
    int32_t profile;         /* 1: launch each sweep's kernels from the host with CUDA events around
                                each one (same kernels and arguments, no graph); read with di_get_profile */
    int32_t select;          /* a di_select value: which nodes a sweep diffuses (default DI_SELECT_REF) */
    int32_t direction;       /* 0: every sweep pushes along the selected nodes' out-links; 1: a sweep
                                pulls along every node's in-links instead when each of the two
                                sweeps before it diffused at least half of all out-links (the same
                                diffusion; the in-link CSR, 12 bytes per link, is built before the
                                first such solve); 2: the same, but the in-link CSR is built only
                                when the first pull is due (the loop pauses for it and resumes
                                where it stopped), so graphs whose sweeps never turn dense pay
                                nothing */
    int32_t scan_wait_polls; /* polls of each bulk-copy wait of the sweep scan, and of the push's
                                staging of hub rows, before the solve stops with DI_ETIMEOUT (0:
                                2^20; a small value makes a watchdog).  A warp or CTA that gave up
                                then waits, with 2^20 polls, for its copies still in flight; if
                                that wait gives up too, copies may land after the kernel returned,
                                and every later call on the graph returns DI_ETIMEOUT until
                                di_free */
} di_solve_opts;

/*
 * Node choice of a threshold sweep.  Section 4.3 compares ALGO-MAX (argmax F)
 * with two variants that divide F by a cost:
 *   ALGO-OP   argmax F_i / ((#in_i + 1)(#out_i + 1))  (#out: a diffusion costs
 *             #out steps; #in: fluid arriving by many links is worth letting
 *             accumulate)
 *   ALGO-OP2  argmax F_i / (#out_i + 1).
 * As threshold sweeps: DI_SELECT_REF diffuses every node with |F_i| > T;
 * DI_SELECT_OP / _OP2 diffuse every node with (float)|F_i| * w_i >
 * (float)(T * s), w_i = 1/((#in_i+1)(#out_i+1)) or 1/(#out_i+1) rounded to
 * FP32, and s the power of two nearest below the mean of w (so that T * s is on
 * the scale of F * w).  With weights the threshold is never raised: after a
 * sweep that diffused something T = min(T, beta R/n), after an empty one T/2.
 * Any choice converges to the same X (Section 2.2); only the number of steps
 * differs.
 */
typedef enum { DI_SELECT_REF = 0, DI_SELECT_OP = 1, DI_SELECT_OP2 = 2 } di_select;

typedef struct {
    double l1_F;           /* exact |F|_1 at the start of the sweep */
    double removed;        /* sum over selected nodes of (1-d)*sent, or sent for dangling ones */
    double R;              /* residual after the sweep: l1_F - removed */
    double T;              /* threshold the sweep used */
    int64_t sources;       /* nodes selected */
    int64_t edges;         /* out-links pushed */
    int64_t pushed;        /* selected nodes with at least one out-link (frontier entries) */
    double scan_ms;        /* CUDA-event time of the sweep's scan kernel (profiled solves, else 0) */
    double push_ms;        /* CUDA-event time of the sweep's push kernel (profiled solves, else 0) */
    int32_t pull;          /* 1: the sweep pulled along the in-links (di_solve_opts.direction), 0: pushed */
    int32_t pad;
} di_sweep_record;

typedef struct {
    double scan_ms;        /* summed CUDA-event time of the sweep scan kernel */
    double push_ms;        /* summed CUDA-event time of the push kernel */
    double finalize_ms;    /* summed CUDA-event time of the finalize kernel */
    int32_t sweeps;        /* launches of each of the three kernels */
    int32_t pull_sweeps;   /* of those, the sweeps that pulled (push_ms then holds the pull kernel) */
} di_profile;

/* ------------------------------------------------------------------ graphs */

/*
 * Build a device-resident graph for the problem X = dPX + (1-d)V (Section 2.1).
 *   n        number of nodes, 1 <= n < 2^31 - 1
 *   row_ptr  host or device, int32[n+1]; row_ptr[0] = 0, non-decreasing,
 *            row_ptr[n] = nnz
 *   col_idx  host or device, int32[nnz]; every entry in [0, n)
 *   nnz      number of edges, 0 <= nnz < 2^31
 *   d        damping factor, 0 < d < 1 (d = 1 is the non-terminating case the
 *            paper contrasts with, Section 2.2 remark)
 *   V        host or device, double[n], V >= 0, finite, |V|_1 = 1 within 1e-12;
 *            NULL means the uniform vector 1/n (not stored)
 *   stream   a cudaStream_t to issue all work on; NULL means the legacy default
 *            stream
 * The library validates everything on the device and builds, with its own
 * kernels: out-degrees, the in-link lists used by di_power, and the degree
 * bins.  On failure *out is NULL and nothing is leaked.
 */
di_status di_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int64_t nnz, double d,
                          const double *V, void *stream, di_graph **out);

/* Release a graph and all of its device memory.  NULL is allowed. */
void di_free(di_graph *g);

/* n, nnz and d of a graph (any pointer may be NULL). */
di_status di_graph_info(const di_graph *g, int32_t *n, int64_t *nnz, double *d);

/*
 * Copy derived structures to caller buffers (host or device), for checks.  The
 * library numbers nodes internally: the hot targets (di_graph_hot_targets) come
 * first, in that order, then every other node in input order.  Every array
 * below except perm is in that internal numbering.
 *   perm     int32[n]: perm[r] = input id of internal node r
 *   outdeg   int32[n]
 *   in_ptr   int32[n+1], in_src int32[nnz]: in-link lists, sources ascending
 *   bin_of   int32[n]: out-degree bin (0 dangling, 1..3 by the cut values)
 *   in_bin_of int32[n]: in-degree class (0: <= in_cut1 in-links, 1: <= in_cut2, 2: above)
 *   cuts     int32[4]: {out_cut1, out_cut2, in_cut1, in_cut2}; the out-degree cutoffs are the
 *            graph's current ones (8 and 1024 at creation; the autotuners may change them)
 * Any pointer may be NULL to skip that array.  Inputs (V, seeds) and outputs
 * (H, F, X) of every other call are in the caller's numbering.
 */
di_status di_graph_export(const di_graph *g, int32_t *perm, int32_t *outdeg, int32_t *in_ptr, int32_t *in_src,
                          int32_t *bin_of, int32_t *in_bin_of, int32_t *cuts);

/*
 * The hot targets of a graph: the (at most 256) nodes with the largest
 * in-degree, at least 32, ties broken by the lower id, in that order.  The push
 * kernel sums the fluid sent to them in shared memory before adding it to F.
 *   ids    host or device int32[256] (may be NULL); *count receives how many
 */
di_status di_graph_hot_targets(const di_graph *g, int32_t *ids, int32_t *count);

/* ------------------------------------------------------------------ solves */

/*
 * D-iteration with threshold sweeps (ALGO-REF with the dangling-node rule,
 * Sections 2.2 and 3.3; sweeps per Section 4.2).  Each sweep selects
 * S = {i : F_i > T} on a snapshot of F, moves F_i into H_i for all of S, then
 * pushes d*F_i/outdeg_i along every out-link of every i in S (dangling nodes
 * push nothing).  T = beta*R/n, halved after a sweep that selects nothing.
 * The loop stops when R/(1-d) <= tol and the exact |F|_1 confirms it.
 *   H_out  host or device double[n] (caller-owned), receives H (or H/|H|_1)
 *   st     may be NULL
 * Returns DI_ENOTCONVERGED (with H_out and st filled) if a limit hit first.
 */
di_status di_solve(di_graph *g, double tol, int64_t max_edge_pushes, di_prec prec, double *H_out, int normalize,
                   di_stats *st);

/* di_solve with every option (defaults when opts fields are zero, see di_solve_opts). */
di_status di_solve_ex(di_graph *g, const di_solve_opts *opts, double *H_out, di_stats *st);

/*
 * Autotuner.  Solves g to base->tol (base->prec, limits, V) once per candidate
 * and keeps the fastest by device time:
 *   beta              0.125, 0.25, 0.5, 1, 2 (the threshold schedule T = beta R/n;
 *                     the paper only says the threshold is lowered progressively)
 *   select            DI_SELECT_REF, _OP, _OP2 (Section 4.3)
 *   push_ctas_per_sm  2, 4, 8 (the push grid; never below the scan grid)
 *   direction         0, 1 (push only, or pull on dense sweeps)
 * every combination of these, then, with the fastest of them, the cutoffs of the
 * out-degree classes (cut1, cut2): a node with at most cut1 out-links is pushed by
 * one thread, up to cut2 by a half-warp, and above that its row is cut into chunks
 * spread over the CTAs; candidates (8, 1024) (the creation default), (4, 1024),
 * (8, 256), (8, 4096) and (4, 256).
 * Every candidate's result is a valid solve (any choice converges, Section 2.2);
 * only the time differs.  The winning push_ctas_per_sm and cutoffs stay set on g
 * (the cutoffs are shared with di_query_batch and the server); beta, select and
 * direction are returned for the caller to pass in di_solve_opts.
 *   best    receives the fastest candidate
 *   tried   host di_tune_result[cap] (may be NULL): every candidate in the order tried;
 *           *ntried receives their number
 */
typedef struct {
    double beta;
    int32_t select;
    int32_t push_ctas_per_sm;
    double ms;               /* device time of the candidate's solve; -1 if it stopped at a limit */
    int64_t edges_pushed;
    int32_t sweeps;
    int32_t direction;       /* di_solve_opts.direction of the candidate */
    int32_t cut1;            /* out-degree class cutoffs of the candidate */
    int32_t cut2;
} di_tune_result;

di_status di_autotune(di_graph *g, const di_solve_opts *base, di_tune_result *best, di_tune_result *tried,
                      int32_t cap, int32_t *ntried);

/*
 * Autotuner of the batched personalized queries (di_query_batch) for the width of
 * a batch of k queries.  Runs the batch (k, seed_ptr, seeds, w as for
 * di_query_batch, per-query bound tol) once per candidate and keeps the fastest by
 * device time, one setting at a time in this order, each with the best of the ones
 * before it (a coordinate search):
 *   cut1, cut2     the out-degree class cutoffs, as for di_autotune
 *   beta           0.25, 0.5, 1 (T_q = beta R_q / n)
 *   pull_share     2, 4, 8, 16: a sweep is dense (the next one pulls) when its
 *                  selected nodes hold at least L / pull_share out-links
 *   push_ctas_per_sm  2, 4, 8 (grid of the batched push and pull)
 *   lanes          the narrowest row that holds k queries (4, 8, 16, 32 or 64), or
 *                  the next wider one
 * Every candidate is a complete batch; a candidate whose queries do not all reach
 * tol never wins.  The winners stay set on g for batches of that width: later
 * di_query_batch calls with the same lane width use them (a cache per graph and
 * width; the cutoffs are shared with single solves and the server).
 *   best   receives the fastest candidate; tried/cap/*ntried as for di_autotune.
 * Errors: DI_EINVAL for the batch arguments as di_query_batch, DI_ENOTCONVERGED if
 * no candidate converged.
 */
typedef struct {
    double beta;
    double ms;               /* device time of the candidate's batch; -1 if a query stopped at a limit */
    double max_bound;        /* largest per-query bound |F_q|_1/(1-d) of the candidate */
    int64_t edges_pushed;
    int32_t sweeps;
    int32_t lanes;           /* row width the batch ran with */
    int32_t pull_share;
    int32_t push_ctas_per_sm;
    int32_t cut1;
    int32_t cut2;
} di_batch_tune_result;

di_status di_autotune_batch(di_graph *g, int32_t k, const int32_t *seed_ptr, const int32_t *seeds, const double *w,
                            double tol, di_batch_tune_result *best, di_batch_tune_result *tried, int32_t cap,
                            int32_t *ntried);

/*
 * Continue a solve after the graph changed (Section 3.2, updating equation).
 * g_old holds the state (F_n0, H_n0) of its last FP64 solve on P, stopped at any
 * bound; g_new is the updated graph P' (same n and d).  The solve continues on
 * P' from the injected fluid F_0' = F_n0 + d(P' - P)H_n0 and the history H_n0;
 * its limit solves X = dP'X + F_0 with the old F_0 = (1-d)V (the theorem after
 * Theorem 3), so only the change is diffused.  The injected fluid can be
 * negative: sweeps select on |F_i|, R decreases by (1-d)|sent| and stays an
 * upper bound on |F|_1, and st->bound = |F|_1/(1-d) is still a bound on
 * |X - H|_1 since |(I - dP')^-1|_1 <= 1/(1-d).  The new state is kept in g_new,
 * which can then be updated in turn.  g_old == g_new continues the same solve.
 *   opts   tol, beta, limits, trace, profile, select as for di_solve_ex;
 *          prec must be DI_FP64
 *   H_out  host or device double[n]: H_n0 + H'
 * g_old is read; nothing of it changes.
 */
di_status di_solve_update(di_graph *g_old, di_graph *g_new, const di_solve_opts *opts, double *H_out,
                          di_stats *st);

/*
 * Personalized query: di_solve with V replaced by the seed distribution
 * (Section 2.1: V is the personalization vector), V_s = w_s / sum(w) on the
 * seeds and 0 elsewhere.
 *   seeds   host or device int32[nseeds], distinct ids in [0, n)
 *   w       host or device double[nseeds] >= 0 with positive sum; NULL = uniform
 */
di_status di_query(di_graph *g, const int32_t *seeds, const double *w, int32_t nseeds, double tol, di_prec prec,
                   double *H_out, di_stats *st);

/*
 * Up to 64 personalized queries solved together (Section 2.1: V is the
 * personalization vector; each query has its own V_q).  Their fluids share one
 * interleaved FP32 row per node (4, 8, 16, 32 or 64 lanes, the narrowest that
 * holds k; 4 bytes per lane), so each read of a node's
 * out-links serves every query; histories are FP64.  A sweep selects node i when
 * some query that has not stopped has F_q[i] > T_q (T_q = 0.5 R_q/n), moves the
 * whole row into H and diffuses it along the out-links: pushed, or, after a sweep
 * whose selected nodes held at least a quarter of all out-links (rows of 8 lanes
 * or more), gathered target by target along the in-links (the same diffusion).
 * Each query stops when its own |F_q|_1/(1-d) <= tol, confirmed in FP64.
 *   k         1 <= k <= 64 queries
 *   seed_ptr  host or device int32[k+1]: query q's seeds are seeds[seed_ptr[q] ..
 *             seed_ptr[q+1]), at least one each (duplicates add their weights)
 *   seeds     host or device int32[seed_ptr[k]], ids in [0, n)
 *   w         host or device double[seed_ptr[k]] >= 0 (NULL: uniform over each
 *             query's seeds); each query's weights need a positive sum
 *   H_out     host or device double[k][n]: query q's H at H_out[q*n .. q*n+n)
 *   st_q      host di_stats[k] (may be NULL): per-query bound and convergence
 *   st_all    host di_stats (may be NULL): sweeps, pushed out-links (each serves
 *             all k queries), device seconds
 */
di_status di_query_batch(di_graph *g, int32_t k, const int32_t *seed_ptr, const int32_t *seeds, const double *w,
                         double tol, double *H_out, di_stats *st_q, di_stats *st_all);

/*
 * di_query_batch (the same computation, Section 2.1) with a profiling switch.
 * profile = 1 launches each sweep's kernels (scan, push, pull, finalize) from
 * the host with CUDA events around them, instead of the captured loop (the same
 * kernels and arguments), and fills *prof (host): scan_ms, push_ms (the push and
 * pull kernels of each sweep together), finalize_ms, sweeps, pull_sweeps.
 * profile = 0 is di_query_batch; prof may then be NULL.  Errors: those of
 * di_query_batch, and DI_EINVAL for profile not 0 or 1, or profile = 1 with
 * prof NULL.
 */
di_status di_query_batch_ex(di_graph *g, int32_t k, const int32_t *seed_ptr, const int32_t *seeds, const double *w,
                            double tol, int32_t profile, double *H_out, di_stats *st_q, di_stats *st_all,
                            di_profile *prof);

/*
 * Power iteration on the uncompleted P (MAT-ITER, Section 4): X_0 = 0,
 * X_{k+1} = dPX_k + (1-d)V, computed by a pull over in-links; stops when
 * |X_{k+1} - X_k|_1 * d/(1-d) < tol (the paper's rule).  FP64.
 *   X_out  host or device double[n]
 * st->sweeps counts products, st->edges_pushed = products * nnz.
 */
di_status di_power(di_graph *g, double tol, int32_t max_iter, double *X_out, di_stats *st);

/*
 * di_power with a profiling switch.  profile = 1 launches each product's two
 * kernels (pull, finalize) from the host with CUDA events around each, instead
 * of the captured graph loop; the summed event times are written to *pull_ms and
 * *finalize_ms (either may be NULL).  Results are identical to di_power.
 */
di_status di_power_ex(di_graph *g, double tol, int32_t max_iter, int32_t profile, double *X_out, di_stats *st,
                      double *pull_ms, double *finalize_ms);

/*
 * Per-sweep records of the last solve made with opts.trace = 1.
 *   out  host di_sweep_record[cap]; *count receives the number available
 *        (records beyond cap are not copied).
 */
di_status di_get_trace(const di_graph *g, di_sweep_record *out, int32_t cap, int32_t *count);

/*
 * Current fluid F and history H of the last D-iteration solve (FP64 copies,
 * host or device double[n] each; either may be NULL).  With the residual they
 * are the complete state (Theorem 1: H + F = F_0 + dPH), used by checks.
 */
di_status di_get_state(const di_graph *g, double *F_out, double *H_out);

/*
 * Load a saved state (F, H) into the graph: the resume half of a checkpoint
 * whose save half is di_get_state.  The state must satisfy Theorem 1 on this
 * graph, H + F = F_0 + dPH with F_0 = (1-d)V: the call computes the residual
 * Z = F_0 - H - F + dPH and accepts the state only when
 *   max_j |Z_j| <= rtol * max_j (|H_j| + |F_j| + F_0,j).
 * A state kept by a global solve (di_solve, di_solve_ex, di_solve_update) of
 * this graph, or of a graph with the same nodes, links, V and d, satisfies it
 * up to rounding (about 1e-14 relative in FP64; an FP32-mixed state about 1e-7);
 * a query's state does not, as its F_0 is the query's.
 *   F_in, H_in  host or device double[n] each, in the caller's numbering; both
 *               required.  The call reads them and keeps no pointer.
 *   rtol        accepted relative deviation (>= 0)
 *   deviation   host double*, may be NULL: receives the relative deviation,
 *               also when the state is rejected
 * On success the graph's FP64 state becomes (F, H), as if its last FP64 solve
 * had stopped there: di_solve_update(g, g, ...) continues it to a new bound, and
 * di_get_state returns it.  Returns DI_EINVAL, with the graph's state unchanged,
 * for a NaN or an infinity in F or H or a deviation above rtol.  It allocates
 * device scratch of 3 double[n] (plus a copy of each host input) for the call.
 */
di_status di_set_state(di_graph *g, const double *F_in, const double *H_in, double rtol, double *deviation);

/*
 * The debug build (libditer_debug.so, compiled with DI_DEBUG) checks the indices its sweep
 * kernels compute before using them: list appends of the scan against their warp's region,
 * list positions and node ids read by the push, pushed-to columns and pull link endpoints
 * against [0, n).  A failed check records its first failure in a device word and skips the
 * access (it never traps); the solve, query or update then returns DI_EKERNEL naming the
 * check and the index.  The release build compiles none of it.
 *   di_debug_build     1 in the debug build, 0 in the release build
 *   di_debug_selftest  the debug build records one failure (code 99, index 12345) from a
 *                      kernel that touches no memory and reports it: returns DI_EKERNEL and
 *                      writes the recorded word, (99 << 48) | 12345, to *word (may be NULL).
 *                      The release build returns DI_EINVAL.
 */
int32_t di_debug_build(void);
di_status di_debug_selftest(uint64_t *word);

/*
 * Per-kernel device times of the last solve made with opts.profile = 1.
 *   out  host di_profile*
 */
di_status di_get_profile(const di_graph *g, di_profile *out);

/*
 * Serving: a continuous stream of personalized queries over several graphs.
 *
 * Personalized PageRank (Section 2.1: V is the personalization vector) solved
 * by threshold sweeps (Section 4.2) on interleaved query lanes, as in
 * di_query_batch; queries on one graph share one read of each out-link list.
 * The diffusions of different queries are independent and any order of
 * diffusions reaches the same limit (Section 2.2), so a query gives the same
 * answer (within the two bounds) whether it runs alone or among others, and
 * lanes can be reused mid-flight: between two rounds of sweeps, queries that
 * met their bound leave their lanes and queued queries take them, while the
 * other lanes carry on.
 *
 * Each graph gets a lane pool of 8, 16, 32 or 64 lanes; a lane costs about
 * 16 bytes per node (FP32 fluid, FP64 history, FP32 sweep copy).  Queries take
 * the lowest free lanes, and each round runs on rows of 4, 8, 16, 32 or 64 lanes,
 * the narrowest that covers every busy lane, so light load moves short rows.
 * The pools are sized at creation by di_plan_lanes under mem_budget bytes.
 * Each pool runs on its own CUDA stream, so rounds of different graphs overlap;
 * smaller graphs get higher stream priorities, so their short rounds are not
 * queued behind the long rounds of large graphs.
 *
 * The server is driven from one host thread: di_server_submit queues, and
 * di_server_poll does all the work (finishing rounds, copying results out,
 * admitting queued queries, launching the next rounds) and returns finished
 * queries.  Nothing runs between polls except the rounds already launched.
 */
typedef struct di_server di_server; /* opaque; owns its lane pools and streams */

typedef struct {
    int64_t ticket;       /* returned by di_server_submit */
    int32_t graph;        /* index of the graph in di_server_create's list */
    int32_t status;       /* DI_OK, or DI_ENOTCONVERGED if the lane's sweep limit stopped it */
    double bound;         /* exact |F_q|_1/(1-d) when it stopped: |X_q - H_q|_1 <= bound */
    int32_t sweeps;       /* sweeps the query took part in */
    int32_t lane;         /* lane it ran in */
    double t_submit;      /* di_clock() at di_server_submit */
    double t_admit;       /* di_clock() when it was given a lane */
    double t_done;        /* di_clock() when its H was in the caller's buffer */
} di_completion;

/*
 * Lane counts under a memory budget (host only, no GPU needed).
 *   lane_bytes[i]   bytes one lane of graph i costs; fixed_bytes[i] the rest of its pool
 *   lanes_out[i]    receives 64, 32, 16 or 8
 * Every graph starts at 64 lanes; while the total is above budget, the graph whose
 * lanes cost the most (lowest index on ties) is halved, down to 8.  DI_ENOMEM if
 * 8 lanes each do not fit.
 */
di_status di_plan_lanes(const int64_t *lane_bytes, const int64_t *fixed_bytes, int32_t ngraphs, int64_t budget,
                        int32_t *lanes_out);

/*
 * Create a server over ngraphs graphs (not owned; they must outlive the server and
 * must not be used by other calls while it exists).
 *   mem_budget    device bytes the lane pools may take (<= 0: no limit, 64 lanes each)
 *   round_sweeps  a round returns to the host after this many sweeps at most (1..1024)
 *   lane_sweeps   a query stops with DI_ENOTCONVERGED after this many sweeps (>= 1)
 */
di_status di_server_create(di_graph *const *graphs, int32_t ngraphs, int64_t mem_budget, int32_t round_sweeps,
                           int32_t lane_sweeps, di_server **out);

/* Lanes of each graph's pool (host int32[ngraphs]). */
di_status di_server_lanes(const di_server *s, int32_t *lanes_out);

/*
 * Queue one query on graph `graph`: V uniform over seeds (w == NULL) or
 * proportional to w, stop when |F_q|_1/(1-d) <= tol.
 *   seeds, w  host arrays of nseeds entries (copied at the call)
 *   H_out     NULL (result dropped), device memory, page-locked host memory (written
 *             by the kernel directly), or pageable host memory (staged through the
 *             device); n doubles in input numbering; must stay valid until the query
 *             completes
 *   ticket    receives the query's ticket
 */
di_status di_server_submit(di_server *s, int32_t graph, const int32_t *seeds, const double *w, int32_t nseeds,
                           double tol, double *H_out, int64_t *ticket);

/*
 * Make progress and collect finished queries: returns as soon as at least one
 * query finished, or after wait_s seconds (0: one pass, no waiting).
 *   out   host di_completion[cap]; *nout receives the number written (finished
 *         queries beyond cap are kept for the next call)
 */
di_status di_server_poll(di_server *s, double wait_s, di_completion *out, int32_t cap, int32_t *nout);

/*
 * Withdraw a submitted query.  A queued query is removed at once; a query in a
 * lane stops at the end of the round in flight, and its lane is cleared and
 * given to the next queued query.  Either way the library writes nothing more
 * to the query's H_out (the caller may free it when the call returns) and
 * di_server_poll returns no completion for it.
 *   cancelled  host int32_t*, may be NULL: 1 when the query was withdrawn, 0
 *              when the ticket is not queued or running: it finished (its
 *              completion is, or will be, returned by di_server_poll), was
 *              cancelled before, or was never issued.  The call returns DI_OK
 *              in all these cases.
 */
di_status di_server_cancel(di_server *s, int64_t ticket, int32_t *cancelled);

/* Counters of one graph's lane pool since the server was created. */
typedef struct {
    int64_t rounds;          /* launches of the sweep loop */
    int64_t sweeps;          /* sweeps run; each serves every busy lane */
    int64_t edges_pushed;    /* out-links pushed; each serves every lane of the row */
    int64_t sources_pushed;  /* selected nodes */
    int64_t admitted;        /* queries given a lane */
    int64_t completed;       /* queries copied out */
    int64_t width_sweeps;    /* sum over rounds of sweeps x lanes per row of that round's loop */
    double device_ms;        /* CUDA-event time of the rounds, from lane admission to the lane-state copy */
    int32_t lanes;
    int32_t pad;
    int64_t cancelled;       /* queries withdrawn by di_server_cancel */
} di_server_graph_stats;

di_status di_server_stats(const di_server *s, int32_t graph, di_server_graph_stats *out);

/* Queries queued (no lane yet) and running (in a lane or being copied out). */
di_status di_server_pending(const di_server *s, int64_t *queued, int64_t *running);

/* Waits for launched work, then frees everything; queries not completed are dropped.  NULL-safe. */
void di_server_free(di_server *s);

/* Seconds on the monotonic host clock used for di_completion times. */
double di_clock(void);

/*
 * di_power without any device allocation.  The paper has no counterpart: this
 * is a service for callers that cannot call cudaMalloc -- services that must
 * not grow their device memory after start-up or that hand out memory only
 * from their own pools, plug-ins in a host program that owns the GPU's
 * allocator.  It runs the same power iteration as di_power (X_0 = 0,
 * X_{k+1} = dPX_k + (1-d)/n with the uniform V, stop when
 * |X_{k+1} - X_k|_1 * d/(1-d) < tol) on the caller's device arrays:
 *   n        nodes, 1 <= n <= 65536 (larger n is rejected with DI_EINVAL)
 *   in_ptr   device int32[n+1], in_src device int32[nnz]: the in-link lists
 *            (row j lists every i with an edge i -> j; any order)
 *   row_ptr  device int32[n+1]: the out-link row pointers (out-degrees)
 *   X_out    device double[n], receives X
 * Every array must be device memory of the current GPU (or managed memory);
 * host memory and another GPU's memory are rejected with DI_EINVAL.
 * Its working memory (about 1 MB: two n-sized buffers, partial sums, a control
 * block) is one static array inside the library.  It is committed on a GPU when
 * the library's module for it is loaded there, which with CUDA's lazy module
 * loading is the first call on that GPU; a caller that must not grow its device
 * memory later should make one call during its start-up.  The array then stays
 * until the process exits.  Every call shares that array and it keeps the last
 * call's contents, so calls that overlap on the GPU (two streams, two host
 * threads) race: issue them one after another.  The first call on a device
 * also looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture begins.  The call waits for its stream:
 * after the input checks and after every 16 products it copies a small status
 * block to the host and synchronizes the stream.  The inputs are checked on the
 * device first (DI_EINVAL names the bad array).  Nothing here calls cudaMalloc,
 * cudaFree or any allocating routine.
 */
di_status di_power_noalloc(int32_t n, const int32_t *in_ptr, const int32_t *in_src, int64_t nnz,
                           const int32_t *row_ptr, double d, double tol, int32_t max_iter, double *X_out,
                           di_stats *st, void *stream);

/* Message of the last failure on this host thread ("" if none). */
const char *di_last_error(void);

/* Library version string. */
const char *di_version(void);

/*
 * Self-test of the bounded waits.  Every wait of the sweep scan on a bulk copy
 * gives up after a bounded number of polls, records the failure and returns, so
 * that a copy that never lands stops the solve with DI_ETIMEOUT instead of
 * hanging the GPU.  This call runs that same wait, with `polls` polls (> 0), in
 * `ctas` CTAs (1..1024) on an mbarrier that nothing ever completes, and writes
 * to *gave_up the number of CTAs whose wait ran out (all of them when the
 * mechanism works).  Launched on the default stream; no device memory is left
 * allocated.  Returns DI_EINVAL on bad arguments, DI_ECUDA on a CUDA error.
 */
di_status di_selftest_wait(int32_t polls, int32_t ctas, int32_t *gave_up);

#ifdef __cplusplus
}
#endif

#endif /* DITER_H */
