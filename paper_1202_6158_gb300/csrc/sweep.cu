// sweep.cu -- the D-iteration hot path: threshold sweeps on the device.
//
// One sweep (Section 4.2: every node whose fluid is above a threshold is
// chosen, and the threshold is lowered progressively) is three kernels:
//
//   k_sweep_scan<FT>   reads all of F once (128-bit loads).  It sums |F|_1
//                      exactly in FP64 and selects S = {i : F_i > T}.  For each
//                      selected node it moves the fluid into the history
//                      (H_i += sent, F_i = 0: the J_i F step of Section 2.2), adds
//                      (1-d)*sent to the removed mass (sent for a dangling node,
//                      Section 3.3) and appends {row start, outdeg, d*sent/outdeg}
//                      to the frontier list of the node's out-degree bin.  Lists
//                      are written per scan chunk at offsets fixed at create time,
//                      in ascending id, with no atomics (warp ballot-free scans
//                      of per-thread counts, block prefix through shared memory).
//   k_sweep_push<FT>   one CTA per scan chunk pushes its chunk's frontier:
//                      F_j += d*sent/outdeg_i along every out-link (ALGO-REF's
//                      inner loop) with red.global.add; a CTA per source above
//                      kOutCut2 out-links, a warp per source above kOutCut1, a
//                      thread per source otherwise; column indices come in as
//                      128-bit loads.
//   k_sweep_finalize   one CTA reduces the per-chunk partials in fixed order,
//                      R = |F|_1 - removed, sets the next threshold
//                      T = beta*R/n (halved after an empty sweep), and stops the
//                      CUDA-graph while-loop when R <= tol*(1-d) or a limit hits.
//
// All of S gives its fluid to H before any push (the scan kernel finishes
// before the push kernel starts), so a sweep is the diffusion of the set S on
// a snapshot of F: F' = (I - J_S + dPJ_S)F, H' = H + J_S F.  Theorem 1
// (H + F = F_0 + dPH) holds after every sweep by the induction of Section 3.1.
// Fluid pushed into a node of S during the push stays in F for a later sweep.
//
// The whole loop is one CUDA graph: a while-conditional node whose body is the
// three kernels, so a solve makes no host round trip per sweep.  After the loop
// the exact |F|_1 is recomputed in fixed order to confirm the stop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace diter {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename FT> struct Vec;
template <> struct Vec<double> { using T = double2; static constexpr int N = 2; };
template <> struct Vec<float> { using T = float4; static constexpr int N = 4; };

__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(float *p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// deterministic block sum (256 threads): warp trees then a fixed-order tree of 8 warp sums
template <typename T>
__device__ T block_sum(T v, T *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = T(0);
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// ------------------------------------------------------------------- init

template <typename FT>
__global__ void k_init_state(int n, int npad, FT *__restrict__ F, double *__restrict__ H, const double *__restrict__ V,
                             double one_minus_d) {
    const double u = 1.0 / (double)n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (long long)gridDim.x * blockDim.x) {
        if (i < n) {
            // F_0 = (1-d)V, H_0 = 0 (initialization of ALGO-REF)
            F[i] = (FT)(one_minus_d * (V ? V[i] : u));
            H[i] = 0.0;
        } else {
            F[i] = (FT)0;
        }
    }
}

template <typename FT>
__global__ void k_init_zero(int npad, int n, FT *__restrict__ F, double *__restrict__ H) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (long long)gridDim.x * blockDim.x) {
        F[i] = (FT)0;
        if (i < n) H[i] = 0.0;
    }
}

// F_0 = (1-d) * w_s / sum(w) on the seeds (V of a personalized query)
template <typename FT>
__global__ void k_init_seeds(int nseeds, const int *__restrict__ seeds, const double *__restrict__ w, double wsum,
                             double one_minus_d, FT *__restrict__ F) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nseeds; k += gridDim.x * blockDim.x) {
        double v = (w ? w[k] : 1.0) / wsum;
        atomicAdd(&F[seeds[k]], (FT)(one_minus_d * v));
    }
}

__global__ void k_init_control(SolveState *st, double R0, double tolR, double beta, double one_minus_d, int n,
                               long long max_edges, int max_sweeps, int trace_on) {
    st->R = R0;
    st->tolR = tolR;
    st->beta = beta;
    st->one_minus_d = one_minus_d;
    st->T = beta * R0 / (double)n;
    st->l1_exact = 0.0;
    st->edges = 0;
    st->srcs = 0;
    st->max_edges = max_edges;
    st->sweeps = 0;
    st->max_sweeps = max_sweeps;
    st->trace_on = trace_on;
    st->body_runs = 0;
    // the while-test of ALGO-REF comes first: nothing to do if R/(1-d) <= target already
    st->done = (R0 <= tolR) ? 1 : 0;
}

// ------------------------------------------------------------------- scan

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_sweep_scan(int n, int chunk, FT *__restrict__ F,
                                                             double *__restrict__ H, const int *__restrict__ row_ptr,
                                                             const int *__restrict__ region, int G,
                                                             int *__restrict__ fcount, FEntry *__restrict__ frontier,
                                                             ScanPartial *__restrict__ part,
                                                             const SolveState *__restrict__ st, double d) {
    using VT = typename Vec<FT>::T;
    constexpr int VN = Vec<FT>::N;
    constexpr int NW = kScanThreads / 32;
    __shared__ int s_wcnt[3][NW];
    __shared__ double s_red_d[NW];
    __shared__ long long s_red_l[NW];
    if (st->done) return;
    const double T = st->T;
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long beg = (long long)c * chunk;
    const long long end = min((long long)n, beg + chunk);
    int run0 = region[0 * (G + 1) + c], run1 = region[1 * (G + 1) + c], run2 = region[2 * (G + 1) + c];
    const int start0 = run0, start1 = run1, start2 = run2;
    double l1 = 0.0, removed = 0.0;
    long long edges = 0, srcs = 0, entries = 0;
    const double dd = d, omd = 1.0 - d;

    for (long long t0 = beg; t0 < end; t0 += (long long)kScanThreads * VN) {
        const long long i0 = t0 + (long long)threadIdx.x * VN;
        FT f[VN];
        if (i0 < end) {
            VT v = *reinterpret_cast<const VT *>(F + i0);
            const FT *pv = reinterpret_cast<const FT *>(&v);
#pragma unroll
            for (int k = 0; k < VN; ++k) f[k] = pv[k];
        } else {
#pragma unroll
            for (int k = 0; k < VN; ++k) f[k] = (FT)0;
        }
        int bin[VN];
        FEntry ent[VN];
        bool any = false;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            const long long i = i0 + k;
            const double fv = (double)f[k];
            l1 += fv;
            bin[k] = -1;
            if (i < end && fv > T) {
                any = true;
                srcs += 1;
                H[i] += fv;
                f[k] = (FT)0;
                const int rb = row_ptr[i];
                const int deg = row_ptr[i + 1] - rb;
                if (deg == 0) {
                    removed += fv;
                } else {
                    removed += omd * fv;
                    edges += deg;
                    entries += 1;
                    bin[k] = deg <= kOutCut1 ? 0 : (deg <= kOutCut2 ? 1 : 2);
                    ent[k].beg = rb;
                    ent[k].deg = deg;
                    ent[k].w = (dd * fv) / (double)deg;
                }
            }
        }
        if (any) {
            VT v;
            FT *pv = reinterpret_cast<FT *>(&v);
#pragma unroll
            for (int k = 0; k < VN; ++k) pv[k] = f[k];
            *reinterpret_cast<VT *>(F + i0) = v;
        }
        // ordered compaction of the tile, one bin at a time
        int excl[3], tot[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < VN; ++k) cnt += (bin[k] == b);
            int x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            excl[b] = x - cnt;
            if (lane == 31) s_wcnt[b][w] = x;
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int off = 0, all = 0;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                int v = s_wcnt[b][k];
                off += (k < w) ? v : 0;
                all += v;
            }
            excl[b] += off;
            tot[b] = all;
        }
        __syncthreads();
        int p0 = run0 + excl[0], p1 = run1 + excl[1], p2 = run2 + excl[2];
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            if (bin[k] == 0) frontier[p0++] = ent[k];
            else if (bin[k] == 1) frontier[p1++] = ent[k];
            else if (bin[k] == 2) frontier[p2++] = ent[k];
        }
        run0 += tot[0];
        run1 += tot[1];
        run2 += tot[2];
    }
    if (threadIdx.x == 0) {
        fcount[0 * G + c] = run0 - start0;
        fcount[1 * G + c] = run1 - start1;
        fcount[2 * G + c] = run2 - start2;
    }
    double bl1 = block_sum(l1, s_red_d);
    double brem = block_sum(removed, s_red_d);
    long long bed = block_sum(edges, s_red_l);
    long long bsr = block_sum(srcs, s_red_l);
    long long ben = block_sum(entries, s_red_l);
    if (threadIdx.x == 0) {
        ScanPartial p;
        p.l1 = bl1;
        p.removed = brem;
        p.edges = bed;
        p.srcs = bsr;
        p.entries = ben;
        p.pad = 0;
        part[c] = p;
    }
}

// ------------------------------------------------------------------- push

template <typename FT>
__device__ __forceinline__ void push_row_lanes(const int *__restrict__ col_idx, FT *__restrict__ F, int beg, int deg,
                                               FT w, int lane, int width) {
    // head up to a 16-byte boundary, then int4 loads, then the tail
    const int head = min(deg, (4 - (beg & 3)) & 3);
    for (int t = lane; t < head; t += width) red_add(F + col_idx[beg + t], w);
    const int body = (deg - head) >> 2;
    const int4 *v4 = reinterpret_cast<const int4 *>(col_idx + beg + head);
    for (int k = lane; k < body; k += width) {
        int4 q = __ldg(v4 + k);
        red_add(F + q.x, w);
        red_add(F + q.y, w);
        red_add(F + q.z, w);
        red_add(F + q.w, w);
    }
    const int done = head + 4 * body;
    for (int t = done + lane; t < deg; t += width) red_add(F + col_idx[beg + t], w);
}

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_sweep_push(const int *__restrict__ col_idx, FT *__restrict__ F,
                                                             const int *__restrict__ region,
                                                             const int *__restrict__ fcount, int G,
                                                             const FEntry *__restrict__ frontier,
                                                             const SolveState *__restrict__ st) {
    if (st->done) return;
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // CTA per source: the largest out-degrees
    {
        const int base = region[2 * (G + 1) + c], cnt = fcount[2 * G + c];
        for (int k = 0; k < cnt; ++k) {
            const FEntry e = frontier[base + k];
            push_row_lanes(col_idx, F, e.beg, e.deg, (FT)e.w, threadIdx.x, kScanThreads);
        }
    }
    // warp per source
    {
        const int base = region[1 * (G + 1) + c], cnt = fcount[1 * G + c];
        for (int k = w; k < cnt; k += kScanThreads / 32) {
            const FEntry e = frontier[base + k];
            push_row_lanes(col_idx, F, e.beg, e.deg, (FT)e.w, lane, 32);
        }
    }
    // thread per source
    {
        const int base = region[0 * (G + 1) + c], cnt = fcount[0 * G + c];
        for (int k = threadIdx.x; k < cnt; k += kScanThreads) {
            const FEntry e = frontier[base + k];
            const FT wv = (FT)e.w;
            for (int t = 0; t < e.deg; ++t) red_add(F + __ldg(col_idx + e.beg + t), wv);
        }
    }
}

// --------------------------------------------------------------- finalize

__global__ void k_sweep_finalize(int n, int G, const ScanPartial *__restrict__ part, SolveState *__restrict__ st,
                                 di_sweep_record *__restrict__ trace, cudaGraphConditionalHandle handle,
                                 int in_graph) {
    __shared__ double s_d[8];
    __shared__ long long s_l[8];
    if (st->done) {  // converged before this body ran: leave the loop
        if (threadIdx.x == 0) {
            st->body_runs += 1;
            if (in_graph) cudaGraphSetConditional(handle, 0);
        }
        return;
    }
    double l1 = 0.0, rem = 0.0;
    long long ed = 0, sr = 0, en = 0;
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
        l1 += part[c].l1;
        rem += part[c].removed;
        ed += part[c].edges;
        sr += part[c].srcs;
        en += part[c].entries;
    }
    l1 = block_sum(l1, s_d);
    rem = block_sum(rem, s_d);
    ed = block_sum(ed, s_l);
    sr = block_sum(sr, s_l);
    en = block_sum(en, s_l);
    if (threadIdx.x != 0) return;
    st->body_runs += 1;
    const double Tused = st->T;
    const double R = l1 - rem;  // |F|_1 after the sweep (exact arithmetic)
    st->sweeps += 1;
    st->edges += ed;
    st->srcs += sr;
    if (st->trace_on && st->sweeps <= kTraceCap) {
        di_sweep_record r;
        r.l1_F = l1;
        r.removed = rem;
        r.R = R;
        r.T = Tused;
        r.sources = sr;
        r.edges = ed;
        r.pushed = en;
        trace[st->sweeps - 1] = r;
    }
    st->R = R;
    double Tn = (sr == 0) ? 0.5 * Tused : st->beta * R / (double)n;
    if (!(Tn > 0.0)) Tn = 0.0;
    st->T = Tn;
    int done = 0;
    if (!isfinite(R)) done = 3;
    else if (R <= st->tolR) done = 1;
    else if (st->sweeps >= st->max_sweeps || (st->max_edges > 0 && st->edges >= st->max_edges)) done = 2;
    st->done = done;
    if (done && in_graph) cudaGraphSetConditional(handle, 0);
}

// ----------------------------------------------------------- exact |F|_1

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_l1_partials(int n, int chunk, const FT *__restrict__ F,
                                                              ScanPartial *__restrict__ part) {
    __shared__ double s[8];
    const long long beg = (long long)blockIdx.x * chunk, end = min((long long)n, beg + chunk);
    double a = 0.0;
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) a += fabs((double)F[i]);
    a = block_sum(a, s);
    if (threadIdx.x == 0) part[blockIdx.x].l1 = a;
}

// sum the partials in fixed order; a stop that the exact norm does not confirm resumes
__global__ void k_confirm(int G, int n, const ScanPartial *__restrict__ part, SolveState *__restrict__ st) {
    __shared__ double s[8];
    double a = 0.0;
    for (int c = threadIdx.x; c < G; c += blockDim.x) a += part[c].l1;
    a = block_sum(a, s);
    if (threadIdx.x == 0) {
        st->l1_exact = a;
        if (st->done == 1 && !(a <= st->tolR)) {
            st->done = 0;
            st->R = a;
            st->T = st->beta * a / (double)n;
        }
    }
}

// ---------------------------------------------------------------- outputs

__global__ void k_sum_h(int n, const double *__restrict__ H, double *out_partials) {
    __shared__ double s[8];
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a += H[i];
    a = block_sum(a, s);
    if (threadIdx.x == 0) out_partials[blockIdx.x] = a;
}

__global__ void k_scale_copy(int n, const double *__restrict__ H, const double *__restrict__ partials, int np,
                             double *__restrict__ out) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < np; ++k) a += partials[k];
        inv = a > 0.0 ? 1.0 / a : 0.0;
    }
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = H[i] * inv;
}

template <typename FT>
__global__ void k_to_double(int n, const FT *__restrict__ in, double *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

int elem_grid(di_graph *g, long long work) {
    long long b = (work + 255) / 256;
    return (int)std::max(1LL, std::min(b, (long long)g->num_sms * 8));
}

// Build the while-loop graph of one precision: body = scan -> push -> finalize.
template <typename FT>
di_status build_sweep_graph(di_graph *g, int slot, FT *F) {
    cudaGraph_t graph = nullptr;
    DI_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphConditionalHandleCreate"); }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphAddNode(conditional)"); }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaStreamBeginCaptureToGraph"); }
    k_sweep_scan<FT><<<g->G, kScanThreads, 0, g->cap>>>(g->n, g->chunk, F, g->H, g->row_ptr, g->region, g->G, g->fcount,
                                                         g->frontier, g->part, g->st, g->d);
    k_sweep_push<FT><<<g->G, kScanThreads, 0, g->cap>>>(g->col_idx, F, g->region, g->fcount, g->G, g->frontier, g->st);
    k_sweep_finalize<<<1, 256, 0, g->cap>>>(g->n, g->G, g->part, g->st, g->trace, handle, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(g->cap, &captured);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaStreamEndCapture"); }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphInstantiate(sweeps)"); }
    g->graph[slot] = graph;
    g->exec[slot] = exec;
    return DI_OK;
}

template <typename FT>
di_status solve_impl(di_graph *g, const di_solve_opts &o, FT *F, int slot, const int *seeds, const double *seed_w,
                     int nseeds, double wsum, double *H_out, bool out_dev, di_stats *stats) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    const int npad = g->G * g->chunk;
    const double omd = 1.0 - g->d;
    if (!g->exec[slot]) {
        di_status r = build_sweep_graph<FT>(g, slot, F);
        if (r != DI_OK) return r;
    }
    DI_CUDA(cudaEventRecord(g->ev0, s));
    if (seeds) {
        k_init_zero<FT><<<elem_grid(g, npad), 256, 0, s>>>(npad, n, F, g->H);
        k_init_seeds<FT><<<std::max(1, std::min(1024, (nseeds + 255) / 256)), 256, 0, s>>>(nseeds, seeds, seed_w, wsum,
                                                                                          omd, F);
    } else {
        k_init_state<FT><<<elem_grid(g, npad), 256, 0, s>>>(n, npad, F, g->H, g->V, omd);
    }
    const double beta = o.beta > 0 ? o.beta : 0.5;
    const int max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 1000000;
    k_init_control<<<1, 1, 0, s>>>(g->st, omd, o.tol * omd, beta, omd, n, o.max_edge_pushes, max_sweeps,
                                   o.trace ? 1 : 0);
    DI_CUDA(cudaGetLastError());
    int attempts = 0;
    g->prof = di_profile{};
    for (int attempt = 0; attempt < 8; ++attempt) {
        ++attempts;
        if (o.profile) {
            // same kernels and arguments as the graph body, launched from the host with events around each
            cudaGraphConditionalHandle none = 0;
            for (;;) {
                DI_CUDA(cudaEventRecord(g->pev[0], s));
                k_sweep_scan<FT><<<g->G, kScanThreads, 0, s>>>(n, g->chunk, F, g->H, g->row_ptr, g->region, g->G,
                                                              g->fcount, g->frontier, g->part, g->st, g->d);
                DI_CUDA(cudaEventRecord(g->pev[1], s));
                k_sweep_push<FT><<<g->G, kScanThreads, 0, s>>>(g->col_idx, F, g->region, g->fcount, g->G,
                                                              g->frontier, g->st);
                DI_CUDA(cudaEventRecord(g->pev[2], s));
                k_sweep_finalize<<<1, 256, 0, s>>>(n, g->G, g->part, g->st, g->trace, none, 0);
                DI_CUDA(cudaEventRecord(g->pev[3], s));
                DI_CUDA(cudaGetLastError());
                DI_CUDA(cudaMemcpyAsync(g->h_st, g->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
                DI_CUDA(cudaStreamSynchronize(s));
                float t0 = 0.f, t1 = 0.f, t2 = 0.f;
                DI_CUDA(cudaEventElapsedTime(&t0, g->pev[0], g->pev[1]));
                DI_CUDA(cudaEventElapsedTime(&t1, g->pev[1], g->pev[2]));
                DI_CUDA(cudaEventElapsedTime(&t2, g->pev[2], g->pev[3]));
                g->prof.scan_ms += t0;
                g->prof.push_ms += t1;
                g->prof.finalize_ms += t2;
                g->prof.sweeps += 1;
                if (g->h_st->done != 0) break;
            }
        } else {
            DI_CUDA(cudaGraphLaunch(g->exec[slot], s));
        }
        k_l1_partials<FT><<<g->G, kScanThreads, 0, s>>>(n, g->chunk, F, g->part);
        k_confirm<<<1, 256, 0, s>>>(g->G, n, g->part, g->st);
        DI_CUDA(cudaGetLastError());
        DI_CUDA(cudaMemcpyAsync(g->h_st, g->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        if (g->h_st->done != 0) break;
    }
    DI_CUDA(cudaEventRecord(g->ev1, s));
    // outputs
    if (o.normalize) {
        const int np = elem_grid(g, n);
        double *partials = nullptr;
        DI_CUDA(cudaMallocAsync(&partials, sizeof(double) * (size_t)np, s));
        k_sum_h<<<np, 256, 0, s>>>(n, g->H, partials);
        if (out_dev) {
            k_scale_copy<<<elem_grid(g, n), 256, 0, s>>>(n, g->H, partials, np, H_out);
        } else {
            double *dtmp = nullptr;
            DI_CUDA(cudaMallocAsync(&dtmp, sizeof(double) * (size_t)n, s));
            k_scale_copy<<<elem_grid(g, n), 256, 0, s>>>(n, g->H, partials, np, dtmp);
            DI_CUDA(cudaMemcpyAsync(H_out, dtmp, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(dtmp, s);
        }
        cudaFreeAsync(partials, s);
    } else if (H_out) {
        DI_CUDA(cudaMemcpyAsync(H_out, g->H, sizeof(double) * (size_t)n,
                                out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    DI_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    DI_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    const SolveState &h = *g->h_st;
    if (stats) {
        stats->bound = h.l1_exact / omd;
        stats->l1_F = h.l1_exact;
        stats->R = h.R;
        stats->edges_pushed = h.edges;
        stats->sources_pushed = h.srcs;
        stats->sweeps = h.sweeps;
        stats->converged = h.done == 1 ? 1 : 0;
        stats->seconds = ms * 1e-3;
        // init (2 kernels, 3 for a seeded query) + 3 per loop iteration + 2 per confirmation
        stats->kernel_launches = (seeds ? 3 : 2) + 3LL * h.body_runs + 2LL * attempts;
    }
    if (h.done == 3) return set_error(DI_EKERNEL, "residual became non-finite");
    if (h.done != 1) return set_error(DI_ENOTCONVERGED, "stopped by a limit before |F|_1/(1-d) <= tol");
    return DI_OK;
}

}  // namespace

di_status sweep_alloc(di_graph *g) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    const int npad = g->G * g->chunk;
    const long long cap = std::max<long long>(1, (long long)g->bin_count[1] + g->bin_count[2] + g->bin_count[3]);
    DI_CUDA(cudaMallocAsync(&g->H, sizeof(double) * (size_t)npad, s));
    DI_CUDA(cudaMallocAsync(&g->frontier, sizeof(FEntry) * (size_t)cap, s));
    DI_CUDA(cudaMallocAsync(&g->part, sizeof(ScanPartial) * (size_t)g->G, s));
    DI_CUDA(cudaMallocAsync(&g->st, sizeof(SolveState), s));
    DI_CUDA(cudaMemsetAsync(g->st, 0, sizeof(SolveState), s));
    DI_CUDA(cudaMemsetAsync(g->H, 0, sizeof(double) * (size_t)npad, s));
    DI_CUDA(cudaMallocAsync(&g->trace, sizeof(di_sweep_record) * kTraceCap, s));
    (void)n;
    return DI_OK;
}

static di_status ensure_fluid(di_graph *g, int prec) {
    const int npad = g->G * g->chunk;
    if (prec == DI_FP64 && !g->F64) {
        DI_CUDA(cudaMallocAsync(&g->F64, sizeof(double) * (size_t)npad, g->stream));
        DI_CUDA(cudaMemsetAsync(g->F64, 0, sizeof(double) * (size_t)npad, g->stream));
    }
    if (prec == DI_FP32_MIXED && !g->F32) {
        DI_CUDA(cudaMallocAsync(&g->F32, sizeof(float) * (size_t)npad, g->stream));
        DI_CUDA(cudaMemsetAsync(g->F32, 0, sizeof(float) * (size_t)npad, g->stream));
    }
    return DI_OK;
}

di_status run_solve(di_graph *g, const di_solve_opts &o, const int *seeds, const double *seed_w, int nseeds,
                    double wsum, double *H_out, bool out_dev, di_stats *st) {
    di_status r = ensure_fluid(g, o.prec);
    if (r != DI_OK) return r;
    g->last_prec = o.prec;
    g->last_trace_on = o.trace ? 1 : 0;
    if (o.prec == DI_FP64)
        return solve_impl<double>(g, o, g->F64, 0, seeds, seed_w, nseeds, wsum, H_out, out_dev, st);
    return solve_impl<float>(g, o, g->F32, 1, seeds, seed_w, nseeds, wsum, H_out, out_dev, st);
}

di_status copy_state(const di_graph *g, double *F_out, bool F_dev, double *H_out, bool H_dev) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    if (F_out) {
        if (g->last_prec == DI_FP32_MIXED && g->F32) {
            double *tmp = nullptr;
            DI_CUDA(cudaMallocAsync(&tmp, sizeof(double) * (size_t)n, s));
            k_to_double<float><<<std::max(1, std::min(1216, (n + 255) / 256)), 256, 0, s>>>(n, g->F32, tmp);
            DI_CUDA(cudaMemcpyAsync(F_out, tmp, sizeof(double) * (size_t)n,
                                    F_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(tmp, s);
        } else if (g->F64) {
            DI_CUDA(cudaMemcpyAsync(F_out, g->F64, sizeof(double) * (size_t)n,
                                    F_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        } else {
            return set_error(DI_EINVAL, "no solve has run on this graph");
        }
    }
    if (H_out)
        DI_CUDA(cudaMemcpyAsync(H_out, g->H, sizeof(double) * (size_t)n,
                                H_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

}  // namespace diter
