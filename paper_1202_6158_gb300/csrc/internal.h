// internal.h -- private structures of libditer shared by its translation units.
//
// Device layout of one graph (n nodes, L edges), all owned by di_graph:
//   perm    int32[n], new_of int32[n]           internal numbering: nodes sorted by in-degree, largest
//                                               first (stable); perm[r] = input id of internal node r,
//                                               new_of = its inverse.  Every array below is indexed by
//                                               internal ids; inputs and outputs are mapped at the edges.
//   row_ptr int32[n+1], col_idx int32[L]        out-link CSR in internal ids
//   hot_ids int32[n_hot]                        input ids of the hot targets = internal 0..n_hot-1
//   in_ptr  int32[n+1], in_src  int32[L]        in-link CSR, sources ascending
//   bin_of  int32[n], cls uint8[npad]           out-degree class (0 dangling, 1 thread, 2 warp, 3 hub
//                                               row; a hub's class byte is 2 + its chunk count)
//   F64 / F32  [n padded to 4]                  fluid F (one of the two per solve)
//   H       double[n]                           history H
//   sel     Sel[n]                              per-sweep selected nodes (id, sent); list L of
//                                               warp sub-chunk g is written at region[L][g] + k
//   X, Z[2]  double[n]                          power-iteration iterate and d*x/outdeg
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/diter.h"

namespace diter {

// ------------------------------------------------------------------ tunables
constexpr int kScanThreads = 256;       // threads of the sweep scan / push CTAs
constexpr int kScanVec = 2;             // fluid elements per thread per tile (16 B of FP64)
constexpr int kScanTile = kScanThreads * kScanVec;
constexpr int kWarps = kScanThreads / 32;  // warps per scan / push CTA; each owns a sub-chunk
constexpr int kStep = 256;              // nodes a warp reads per step (8 per lane)
constexpr int kChunkAlign = kWarps * kStep;  // scan chunks are multiples of 8 warp steps
constexpr int kLists = 4;               // selected nodes: 0 dangling, 1 thread, 2 warp, 3 chunked hub rows
constexpr int kChunkRow = kLists;       // row of fcount / pre holding each sub-chunk's hub chunk count
constexpr int kCountRows = kLists + 1;  // rows of fcount / pre: the lists, then the hub chunks
constexpr int kMaxScanBlocks = 152 * 8; // 8 CTAs per SM on 152 SMs
constexpr int kOutCut1 = 8;             // out-degree <= cut1: one thread per source
constexpr int kOutCut2 = 1024;          // out-degree <= cut2: one warp per source; above: whole CTA
constexpr int kInCut1 = 8;              // in-degree classes reported by di_graph_export: <= cut1,
constexpr int kInCut2 = 2048;           // <= cut2, above
constexpr int kTraceCap = 4096;         // sweep records kept when tracing
constexpr int kExactEvery = 4;          // the scan sums |F|_1 exactly every this many sweeps
constexpr int kHubChunk = 1024;         // out-links per chunk of a hub row (class 3) in the push
constexpr int kMaxHubChunks = 253;      // chunks of one hub row at most (its class byte is 2 + chunks)
constexpr int kColPad = 4;              // zero ints allocated past the last column index
constexpr int kHotSlots = 256;          // most-linked-to targets accumulated in shared memory by the push
constexpr int kHotMinInDeg = 32;        // a target needs at least this many in-links to get a slot

// one selected node of a sweep that has out-links, and the fluid it hands over
template <typename FT>
struct __align__(16) Sel {
    int node;
    int pad;
    FT sent;    // F_node at the snapshot, in the fluid's precision
};

// a node's out-link range and d/outdeg, read by the push with one 16-byte access
template <typename FT>
struct __align__(16) RowRec {
    int beg;
    int deg;
    FT inv;
};

// per-CTA results of the sweep scan, reduced in fixed order by the finalize kernel.
// Fluid sums are 64-bit fixed point at the sweep's scale 2^-S (see fixed_scale).
struct __align__(16) ScanPartial {
    long long l1;      // sum of F over the CTA's chunk before selection (fixed point)
    long long out;     // fluid of selected nodes with children (fixed point)
    long long dng;     // fluid of selected dangling nodes (fixed point)
    long long edges;   // out-links of the selected nodes (written by the push kernel)
    long long srcs;    // selected nodes
    long long entries; // selected nodes with out-links
    double l1d;        // FP64 sum, used by the exact confirmation kernel
    long long err;     // 1: a bulk-copy wait of the scan gave up (the solve stops with DI_ETIMEOUT)
};

// device-resident control block of one solve
struct SolveState {
    double R;              // residual after the last sweep
    double T;              // threshold of the next sweep
    double tolR;           // stop when R <= tolR (= tol * (1 - d))
    double beta;
    double one_minus_d;
    double l1_exact;       // exact |F|_1 written by the confirmation kernel
    long long edges;       // cumulative out-links pushed
    long long srcs;        // cumulative selected nodes
    long long max_edges;
    int sweeps;
    int max_sweeps;
    int done;              // 0 running, 1 converged, 2 limit reached, 3 non-finite residual, 4 scan wait timed out
    int trace_on;
    int body_runs;         // executions of the finalize kernel (one per sweep of a loop iteration)
    int exact;             // 1 when the sweep now running sums |F|_1 exactly (every kExactEvery sweeps)
    int weighted;          // ALGO-OP / OP2 selection: the threshold is never raised
    int pull;              // this sweep's direction: 0 push from the class lists, 1 pull along the in-links
    double wscale;         // weighted selection: the threshold of F*w is T * wscale
    long long pull_edges;  // a sweep that diffused at least this many out-links is dense
    int dense;             // the last sweep was dense: a second dense sweep makes the next one pull
    int wait_polls;        // polls of each bulk-copy wait of the scan before the solve gives up
    int pause_pull;        // the in-link CSR is not built yet: a due pull stops the loop (done = 5) instead
    int undrained;         // a timed-out scan warp returned with bulk copies possibly still landing
    int n;                 // nodes (read by the index checks of the DI_DEBUG build)
};

// batched personalized queries: up to kLanes queries interleaved in one fluid row
// captured sweep loops: 7 selection / precision variants, each push-only or with the pull direction
constexpr int kSweepSlots = 14;
// a sweep is dense when its selected nodes hold at least 1/kPullShareBatch (batch) or
// 1/kPullShareSolve (single solve) of all out-links; a batch pulls after one dense sweep, a
// single solve after two in a row (one FP64 pull sweep costs about as much as pushing 0.7 L
// out-links)
constexpr long long kPullShareBatch = 4;
constexpr long long kPullShareSolve = 2;

constexpr int kLanes = 64;              // queries per batch (the width of a fluid row)
constexpr int kBatchHot = 32;           // hot targets whose rows the batched push sums in shared memory
constexpr int kWidths = 5;              // row widths of the batched loops: 4, 8, 16, 32, 64 lanes

struct BatchQ {            // per query lane
    double R;              // residual after the last sweep
    double T;              // threshold of the next sweep (+inf once the query has stopped)
    double tolR;           // stop when R <= tolR
    double l1_acc;         // |F_q|_1 summed by the current sweep's scan
    double rem_acc;        // mass removed by the current sweep
    double l1_exact;       // FP64 |F_q|_1 of the confirmation
    int active;            // a query occupies this lane
    int done;              // 0 running, 1 stopped on its bound, 2 stopped at its sweep limit
    int selected;          // lanes of this query above its threshold in the current sweep
    int sweeps;            // sweeps this query has taken part in
    int confirmed;         // the stop was checked against the exact FP64 |F_q|_1
    int pad[3];
};

struct BatchCtl {
    long long edges;       // out-links pushed (each serves all lanes)
    long long srcs;        // selected nodes
    double beta;
    int sweeps;
    int max_sweeps;
    int all_done;          // 1 no lane open, 2 the loop's sweep limit hit
    int body_runs;
    int round_sweeps;      // sweeps of the current launch of the loop
    int round_cap;         // the loop returns after this many sweeps
    int stop_on_done;      // the loop also returns when a lane stops
    int lane_max_sweeps;   // a lane stops (done = 2) after this many sweeps
    int newly;             // a lane stopped in the current launch
    int pull;              // this sweep's direction: 0 push from the selected rows, 1 pull into every row
    long long sel_edges;   // out-links of the sweep's selected nodes, summed by the scan
};

// lanes to free and lanes to start, applied by the kernel that opens a round of the serving loop
struct LaneAdmin {
    unsigned long long retire;
    unsigned long long admit;
    double tolR[kLanes];
};

// lanes whose histories are copied out (and whose columns are cleared) in one launch
struct LaneRetire {
    int count;
    int lane[kLanes];
    double *out[kLanes];   // n doubles each, input numbering; NULL: clear only
};

struct PowerState {
    double delta;          // |X_k - X_{k-1}|_1 of the last product
    double tol;            // stop when delta * d/(1-d) < tol
    double d;
    int iters;
    int max_iters;
    int done;              // 1 stop rule met, 2 limit reached, 3 non-finite
    int cur;               // which Z buffer holds d*X/outdeg of the current iterate
};

struct PowerPartial {
    double delta;
    double pad;
};

// interleaved query lanes with their own sweep scratch: the buffers of di_query_batch,
// and of each graph a serving loop holds
// A hub row (class 3) is pushed in chunks: ceil(deg / kHubChunk) of them, at most kMaxHubChunks,
// of equal length ceil(deg / chunks).  The class byte of a hub node is 2 + its chunk count, so the
// sweep scans count the chunks of the rows they list without reading the row records.
__host__ __device__ inline int hub_chunk_count(int deg) {
    const int c = (deg + kHubChunk - 1) / kHubChunk;
    return c < kMaxHubChunks ? c : kMaxHubChunks;
}
__host__ __device__ inline int hub_chunk_len(int deg, int chunks) { return (deg + chunks - 1) / chunks; }
__host__ __device__ inline int class_of_byte(int c) { return c < 3 ? c : 3; }

// settings of the batched loop for one row width, chosen by di_autotune_batch
struct BatchTune {
    double beta = 0.5;                 // T_q = beta R_q / n
    int pull_share = (int)kPullShareBatch;  // a sweep is dense when its nodes hold >= L / pull_share out-links
    int push_per_sm = 4;               // CTAs per SM of the batched push and pull kernels
    int exec_slot = -1;                // the width to run batches of this width with (-1: the same)
    int tuned = 0;
};

struct BatchPool {
    int cap_lanes = 0;                 // lanes per row the buffers hold
    int stride = 0;                    // floats between rows: 0 = the loop's width (a fresh batch packs its rows);
                                       // a serving pool keeps cap_lanes and runs narrower loops on the low lanes
    long long rows = 0;                // fluid rows (n padded to the scan layout)
    float *Fb = nullptr;               // [rows][K] interleaved fluid, FP32
    double *Hb = nullptr;              // [n][K] histories, FP64
    float *selb_rows = nullptr;        // [n][K] rows of the selected nodes of a sweep
    int *selb_node = nullptr;          // [n]
    int *spos = nullptr;               // [rows] list position of each node selected in the sweep, -1 otherwise
    int *fcount = nullptr, *pre = nullptr;
    unsigned *ticket = nullptr;
    BatchQ *bq = nullptr, *h_bq = nullptr;
    BatchCtl *bctl = nullptr, *h_bctl = nullptr;
    // captured loops for rows of 4, 8, 16, 32, 64 lanes
    cudaGraph_t graph[kWidths] = {};
    cudaGraphExec_t exec[kWidths] = {};
};

}  // namespace diter

struct di_graph {
    int n = 0;
    long long nnz = 0;
    double d = 0.85;
    int dev = 0;
    int num_sms = 152;
    int push_per_sm = 4;               // push CTAs per SM at least (the push grid never shrinks below the scan's)
    int cut1 = diter::kOutCut1, cut2 = diter::kOutCut2;  // out-degree class cutoffs in use (set_out_classes)
    diter::BatchTune btune[diter::kWidths];   // batched-query settings per row width (di_autotune_batch)
    bool untrusted = false;            // a scan wait timed out twice: copies may have landed late (DI_ETIMEOUT)
    cudaStream_t stream = nullptr;     // user stream
    cudaStream_t cap = nullptr;        // private stream used for graph capture

    // graph
    int *row_ptr = nullptr, *col_idx = nullptr;
    int *in_ptr = nullptr, *in_src = nullptr;   // built at first use (build_transpose)
    int *in_dst = nullptr;                      // [L] target of each in-link, built with the first batch pool
    bool transposed = false;
    int *bin_of = nullptr;
    unsigned char *cls = nullptr;      // [npad] out-degree class per node, 0 on the padding
    double *V = nullptr;               // NULL: uniform 1/n
    double *inv_deg = nullptr;         // d / outdeg(i), 0 for dangling nodes (FP64)
    float *inv_deg32 = nullptr;        // the same rounded to FP32
    diter::RowRec<double> *rec64 = nullptr;  // [n] {row start, outdeg, d/outdeg}
    diter::RowRec<float> *rec32 = nullptr;   // [n] the same with d/outdeg in FP32
    int bin_count[4] = {0, 0, 0, 0};   // static out-degree class sizes
    int *hot_ids = nullptr;            // [kHotSlots] input id of each hot target (internal ids 0..n_hot-1)
    int n_hot = 0;
    unsigned long long *rowhash = nullptr;  // [n] fingerprint of each input row (input numbering), at first update
    int *perm = nullptr;               // [n] internal -> input id
    int *new_of = nullptr;             // [n] input -> internal id

    // sweep structures
    int G = 0;                         // scan CTAs
    int chunk = 0;                     // nodes per scan CTA (multiple of kChunkAlign)
    int W = 0;                         // warp sub-chunks, G * kWarps, chunk / kWarps nodes each
    int *region = nullptr;             // [kLists][W+1]: offset of each list's entries per sub-chunk
    int *fcount = nullptr;             // [kCountRows][W]: entries written per sub-chunk in the last sweep, per
                                       // list, then the chunks of the hub rows listed
    int *pre = nullptr;                // kCountRows*(W+1) ints: the two-level list offsets the scan writes,
                                       // [(L-1)G + b] the total of row L in scan CTA b, [L W + g] sub-chunk
                                       // g's offset within its CTA's part (L = 1 .. kCountRows-1)
    void *sel = nullptr;               // Sel<FT>[n]: the selected nodes of a sweep
    double *F64 = nullptr;
    float *F32 = nullptr;
    double *H = nullptr;
    diter::ScanPartial *part = nullptr;
    diter::SolveState *st = nullptr;
    di_sweep_record *trace = nullptr;
    int last_prec = -1;
    int last_trace_on = 0;
    di_profile prof = {};
    float *sweep_ms = nullptr;         // host: [kTraceCap][2] scan and push event times of a profiled solve
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};

    // power iteration
    double *X = nullptr;
    double *Z[2] = {nullptr, nullptr};
    double *Y = nullptr;               // [n] the product being formed: (1-d)V + the gathered z
    diter::PowerPartial *ppart = nullptr;
    diter::PowerState *pst = nullptr;
    double pprof_ms[2] = {0.0, 0.0};   // profiled power iteration: pull, finalize

    // batched queries (allocated at the first batch)
    diter::BatchPool *bp = nullptr;

    // captured solve loops: [0] FP64 sweeps, [1] FP32-mixed sweeps, [2] power iteration,
    // [3 + 2*(select-1) + prec] weighted sweeps (ALGO-OP select 1, ALGO-OP2 select 2)
    cudaGraph_t graph[diter::kSweepSlots] = {};
    cudaGraphExec_t exec[diter::kSweepSlots] = {};
    void *wpull = nullptr;             // [npad] FP64 or FP32: sent * d/outdeg of the nodes a pull sweep selected, else 0
    float *wsel[2] = {nullptr, nullptr};   // [npad] selection weights of ALGO-OP / ALGO-OP2 (0 on the padding)
    double wscale[2] = {1.0, 1.0};         // 2^floor(log2(mean weight))

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    diter::SolveState *h_st = nullptr; // pinned host mirror
    diter::PowerState *h_pst = nullptr;
};

namespace diter {

// error plumbing (api.cu)
di_status set_error(di_status s, const std::string &msg);
di_status cuda_fail(cudaError_t e, const char *what);

// graph ingest (graph_build.cu)
// g->row_ptr holds the CSR's row starts; col_host non-NULL: the caller's host col_idx, copied
// into g->col_idx here in chunks that overlap the in-degree count (else g->col_idx holds it)
di_status build_graph(di_graph *g, const int *col_host);
di_status build_in_dst(di_graph *g);  // the transpose, then in_dst
di_status in_degree_classes(di_graph *g, int *out_dev);
di_status ensure_rowhash(di_graph *g);  // fingerprints of the input rows (graph updates)
di_status selftest_wait(int polls, int ctas, int *gave_up);
di_status build_transpose(di_graph *g);   // the in-link CSR and its bins, at first use
di_status validate_v(di_graph *g, const double *V_dev);

// sweeps (sweep.cu)
di_status sweep_alloc(di_graph *g);
di_status run_solve(di_graph *g, const di_solve_opts &o, const int *seeds_dev, const double *seed_w_dev, int nseeds,
                    double wsum, double *H_out, bool out_on_device, di_stats *st);
// graph update (Section 3.2): continue g_old's FP64 state on g_new
di_status run_update(di_graph *g_old, di_graph *g_new, const di_solve_opts &o, double *H_out, bool out_on_device,
                     di_stats *st);
di_status copy_state(const di_graph *g, double *F_out, bool F_dev, double *H_out, bool H_dev);
di_status gather_x(di_graph *g, const double *src, double *dst, bool dst_dev);

// power iteration (power.cu)
di_status power_alloc(di_graph *g);
di_status run_power(di_graph *g, double tol, int max_iter, int profile, double *X_out, bool out_on_device,
                    di_stats *st);
int scan_blocks_per_sm();

// batched queries (batch.cu)
di_status run_query_batch(di_graph *g, int k, const int *seed_ptr, const int *seeds, const double *w, double tol,
                          double beta, int max_sweeps, double *H_out, bool out_dev, di_stats *st_q, di_stats *st_all,
                          di_profile *prof);  // prof != NULL: the loop launched from the host, timed
di_status pool_alloc(di_graph *g, BatchPool *p, int lanes, cudaStream_t s);
void pool_free(BatchPool *p, cudaStream_t s);
long long pool_bytes(const di_graph *g, int lanes);
di_status pool_build_loop(di_graph *g, BatchPool *p, int slot);
di_status set_out_classes(di_graph *g, int cut1, int cut2);
di_status batch_args(di_graph *g, int k, const int32_t *seed_ptr, const int32_t *seeds, const double *w, double tol,
                     std::vector<int32_t> &hp, std::vector<int32_t> &hs, std::vector<double> &hw);
// row widths 4, 8, 16, 32, 64 lanes are slots 0..4: the narrowest that holds k lanes
inline int lane_slot(int k) { return k <= 4 ? 0 : (k <= 8 ? 1 : (k <= 16 ? 2 : (k <= 32 ? 3 : 4))); }
inline int slot_width(int slot) { return 4 << slot; }
// one round of the serving loop on stream s: free and start lanes, diffuse, confirm stops, copy the lane states back
di_status pool_launch_round(di_graph *g, BatchPool *p, int slot, const LaneAdmin &a, int round_cap, int lane_max,
                            double beta, cudaStream_t s);
di_status pool_seed(di_graph *g, BatchPool *p, int K, int nitems, const int *q_dev, const int *seeds_dev,
                    const double *val_dev, cudaStream_t s);
di_status pool_retire(di_graph *g, BatchPool *p, int K, const LaneRetire &r, cudaStream_t s);
di_status pool_reset(di_graph *g, BatchPool *p, int K, double beta, cudaStream_t s);

// pointer kinds (api.cu): device or host-mapped memory a kernel can write, else pageable host memory
bool is_device_ptr(const void *p);
void *kernel_ptr(void *p);

// helpers
inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
template <typename FT> inline const RowRec<FT> *rec_of(const di_graph *g);
template <> inline const RowRec<double> *rec_of<double>(const di_graph *g) { return g->rec64; }
template <> inline const RowRec<float> *rec_of<float>(const di_graph *g) { return g->rec32; }
template <typename FT> inline Sel<FT> *sel_of(const di_graph *g) { return reinterpret_cast<Sel<FT> *>(g->sel); }

// the push of one sweep on stream s (push.cu)
template <typename FT> void launch_push(di_graph *g, FT *F, cudaStream_t s);
#ifdef DI_DEBUG
// the first failed index check of the sweep kernels since the last call, cleared (0: none)
unsigned long long dbg_take_sweep();
unsigned long long dbg_take_push();
// DI_EKERNEL naming the first failed check, else DI_OK; *word (may be NULL) receives its word
di_status debug_status(unsigned long long *word = nullptr);
// records a failure from a kernel that touches no memory, then reports it
di_status debug_selftest(unsigned long long *word);
#endif
di_status push_setup();
template <typename FT> void launch_pull(di_graph *g, FT *F, cudaStream_t s);

// push CTAs: the pushes scale with edges, not nodes, so small graphs still get push_per_sm CTAs per SM
inline int push_grid(const di_graph *g) {
    const int m = g->push_per_sm * g->num_sms;
    return g->G > m ? g->G : m;
}

}  // namespace diter

#define DI_CUDA(call)                                                 \
    do {                                                              \
        cudaError_t _e = (call);                                      \
        if (_e != cudaSuccess) return diter::cuda_fail(_e, #call);    \
    } while (0)
