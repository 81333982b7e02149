// power.cu -- MAT-ITER, the plain comparison (Section 4): X_0 = 0,
// X_{k+1} = dPX_k + (1-d)V on the uncompleted P, stopped when
// |X_{k+1} - X_k|_1 * d/(1-d) < tol.
//
// Each product is a pull ("collection", Section 1) over the in-link lists:
//   y_j = (1-d)V_j + sum_{i -> j} z_i,   z_i = d * x_i / outdeg(i)  (0 if dangling)
// with z of the current iterate kept in one of two buffers so the gather never
// sees a value of the product being formed.  Rows are grouped by in-degree at
// create time: a thread per row up to kInCut1 in-links, a warp per row up to
// kInCut2, and above that chunk tasks of kPullChunk in-links, one warp each,
// whose sums meet in a per-row accumulator.  The per-row epilogue (|y - x|,
// x = y, z = d*y/outdeg) is fused into the pull; one CTA finishes the chunked
// rows, reduces |X_{k+1} - X_k|_1 in fixed order and drives the CUDA-graph
// while-loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace diter {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ double block_sum_d(double v, double *sh) {
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    __syncthreads();
    return r;
}

struct PullArgs {
    int n;
    const int *in_ptr, *in_src, *pull_ids, *long_ids, *long_prefix;
    const double *inv_deg;  // d / outdeg, 0 for dangling nodes
    int cnt0, cnt1, nlong, ntasks;
    int BA, BB;
    const double *V;  // NULL: uniform
    double omd, d, u, omdu;
    double *X, *Z0, *Z1, *Ylong;
    PowerPartial *pp;
    PowerState *pst;
};

__device__ __forceinline__ double v_of(const PullArgs &a, int j) { return a.V ? a.V[j] : a.u; }
// (1-d) V_j
__device__ __forceinline__ double omdv_of(const PullArgs &a, int j) { return a.V ? a.omd * a.V[j] : a.omdu; }

// finish row j with its new value y; returns |y - x_j|
__device__ __forceinline__ double finish_row(const PullArgs &a, double *zn, int j, double y) {
    double dlt = fabs(y - a.X[j]);
    a.X[j] = y;
    zn[j] = y * a.inv_deg[j];
    return dlt;
}

// sum of z over a row of at most kInCut1 in-links: index loads, then gathers, then
// the adds in ascending order
__device__ __forceinline__ double short_row_sum(const PullArgs &a, const double *__restrict__ zc, int b, int e) {
    int s[kInCut1];
#pragma unroll
    for (int t = 0; t < kInCut1; ++t) s[t] = b + t < e ? __ldg(a.in_src + b + t) : -1;
    double z[kInCut1];
#pragma unroll
    for (int t = 0; t < kInCut1; ++t) z[t] = s[t] >= 0 ? zc[s[t]] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < kInCut1; ++t)
        if (s[t] >= 0) acc += z[t];
    return acc;
}

__global__ void __launch_bounds__(256) k_pull(PullArgs a) {
    __shared__ double sh[8];
    if (a.pst->done) return;
    const int cur = a.pst->cur;
    const double *__restrict__ zc = cur ? a.Z1 : a.Z0;
    double *zn = cur ? a.Z0 : a.Z1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double delta = 0.0;
    if ((int)blockIdx.x < a.BA) {
        const long long stride = (long long)a.BA * 256;
        long long r = (long long)blockIdx.x * 256 + threadIdx.x;
        for (; r + stride < a.cnt0; r += 2 * stride) {  // two rows in flight
            const int j0 = a.pull_ids[r], j1 = a.pull_ids[r + stride];
            const int b0 = a.in_ptr[j0], e0 = a.in_ptr[j0 + 1], b1 = a.in_ptr[j1], e1 = a.in_ptr[j1 + 1];
            const double s0 = short_row_sum(a, zc, b0, e0);
            const double s1 = short_row_sum(a, zc, b1, e1);
            delta += finish_row(a, zn, j0, omdv_of(a, j0) + s0);
            delta += finish_row(a, zn, j1, omdv_of(a, j1) + s1);
        }
        if (r < a.cnt0) {
            const int j = a.pull_ids[r];
            delta += finish_row(a, zn, j, omdv_of(a, j) + short_row_sum(a, zc, a.in_ptr[j], a.in_ptr[j + 1]));
        }
    } else if ((int)blockIdx.x < a.BA + a.BB) {
        const long long wid = (long long)(blockIdx.x - a.BA) * 8 + w, nw = (long long)a.BB * 8;
        for (long long r = wid; r < a.cnt1; r += nw) {
            const int j = a.pull_ids[a.cnt0 + r];
            const int b = a.in_ptr[j], e = a.in_ptr[j + 1];
            double acc = 0.0;
            for (int k = b + lane; k < e; k += 32) acc += zc[a.in_src[k]];
            acc = warp_sum_d(acc);
            if (lane == 0) delta += finish_row(a, zn, j, omdv_of(a, j) + acc);
        }
    } else {
        const int BC = gridDim.x - a.BA - a.BB;
        const long long wid = (long long)(blockIdx.x - a.BA - a.BB) * 8 + w, nw = (long long)BC * 8;
        for (long long t = wid; t < a.ntasks; t += nw) {
            int lo = 0, hi = a.nlong;  // last r with long_prefix[r] <= t
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (a.long_prefix[mid] <= t) lo = mid; else hi = mid;
            }
            const int j = a.long_ids[lo];
            const long long b = (long long)a.in_ptr[j] + (t - a.long_prefix[lo]) * (long long)kPullChunk;
            const long long e = min((long long)a.in_ptr[j + 1], b + kPullChunk);
            double acc = 0.0;
            for (long long k = b + lane; k < e; k += 32) acc += zc[a.in_src[k]];
            acc = warp_sum_d(acc);
            if (lane == 0) atomicAdd(&a.Ylong[lo], acc);
        }
    }
    delta = block_sum_d(delta, sh);
    if (threadIdx.x == 0) a.pp[blockIdx.x].delta = delta;
}

__global__ void k_power_finalize(PullArgs a, int nparts, cudaGraphConditionalHandle handle, int in_graph) {
    __shared__ double sh[8];
    if (a.pst->done) {
        if (threadIdx.x == 0 && in_graph) cudaGraphSetConditional(handle, 0);
        return;
    }
    const int cur = a.pst->cur;
    double *zn = cur ? a.Z0 : a.Z1;
    double delta = 0.0;
    for (int r = threadIdx.x; r < a.nlong; r += blockDim.x) {
        const int j = a.long_ids[r];
        delta += finish_row(a, zn, j, a.Ylong[r]);
        a.Ylong[r] = omdv_of(a, j);
    }
    delta = block_sum_d(delta, sh);
    double parts = 0.0;
    for (int c = threadIdx.x; c < nparts; c += blockDim.x) parts += a.pp[c].delta;
    parts = block_sum_d(parts, sh);
    if (threadIdx.x != 0) return;
    PowerState *p = a.pst;
    const double dl = parts + delta;
    p->delta = dl;
    p->iters += 1;
    p->cur = cur ^ 1;
    int done = 0;
    if (!isfinite(dl)) done = 3;
    else if (dl * p->d / (1.0 - p->d) < p->tol) done = 1;
    else if (p->iters >= p->max_iters) done = 2;
    p->done = done;
    if (done && in_graph) cudaGraphSetConditional(handle, 0);
}

__global__ void k_power_init(PullArgs a, double tol, int max_iters) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        a.X[i] = 0.0;
        a.Z0[i] = 0.0;
        a.Z1[i] = 0.0;
    }
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < a.nlong; r += (long long)gridDim.x * blockDim.x)
        a.Ylong[r] = omdv_of(a, a.long_ids[r]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.pst->delta = 0.0;
        a.pst->tol = tol;
        a.pst->d = a.d;
        a.pst->iters = 0;
        a.pst->max_iters = max_iters;
        a.pst->done = 0;
        a.pst->cur = 0;
    }
}

PullArgs make_args(di_graph *g) {
    PullArgs a;
    a.n = g->n;
    a.in_ptr = g->in_ptr;
    a.in_src = g->in_src;
    a.inv_deg = g->inv_deg;
    a.pull_ids = g->pull_ids;
    a.cnt0 = g->in_bin_count[0];
    a.cnt1 = g->in_bin_count[1];
    a.nlong = g->n_long_rows;
    a.long_ids = g->pull_ids + g->in_bin_count[0] + g->in_bin_count[1];
    a.long_prefix = g->long_prefix;
    a.ntasks = g->n_long_tasks;
    a.BA = g->pull_blocks[0];
    a.BB = g->pull_blocks[1];
    a.V = g->V;
    a.omd = 1.0 - g->d;
    a.d = g->d;
    a.u = 1.0 / (double)g->n;
    a.omdu = a.omd * a.u;
    a.X = g->X;
    a.Z0 = g->Z[0];
    a.Z1 = g->Z[1];
    a.Ylong = g->Ylong;
    a.pp = g->ppart;
    a.pst = g->pst;
    return a;
}

int role_blocks(long long work, int per_block, int cap) {
    if (work <= 0) return 0;
    return (int)std::max(1LL, std::min((work + per_block - 1) / per_block, (long long)cap));
}

di_status build_power_graph(di_graph *g) {
    PullArgs a = make_args(g);
    const int nparts = g->pull_blocks[0] + g->pull_blocks[1] + g->pull_blocks[2];
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
    k_pull<<<nparts, 256, 0, g->cap>>>(a);
    k_power_finalize<<<1, 256, 0, g->cap>>>(a, nparts, handle, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(g->cap, &captured);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaStreamEndCapture"); }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphInstantiate(power)"); }
    g->graph[2] = graph;
    g->exec[2] = exec;
    return DI_OK;
}

}  // namespace

di_status power_alloc(di_graph *g) {
    cudaStream_t s = g->stream;
    const int cap = g->num_sms * 8;
    g->pull_blocks[0] = role_blocks(g->in_bin_count[0], 256, cap);
    g->pull_blocks[1] = role_blocks(g->in_bin_count[1], 8, cap);
    g->pull_blocks[2] = role_blocks(g->n_long_tasks, 8, cap);
    const int nparts = std::max(1, g->pull_blocks[0] + g->pull_blocks[1] + g->pull_blocks[2]);
    DI_CUDA(cudaMallocAsync(&g->X, sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->Z[0], sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->Z[1], sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->Ylong, sizeof(double) * (size_t)std::max(1, g->n_long_rows), s));
    DI_CUDA(cudaMallocAsync(&g->ppart, sizeof(PowerPartial) * (size_t)nparts, s));
    DI_CUDA(cudaMallocAsync(&g->pst, sizeof(PowerState), s));
    DI_CUDA(cudaMemsetAsync(g->pst, 0, sizeof(PowerState), s));
    return DI_OK;
}

di_status run_power(di_graph *g, double tol, int max_iter, int profile, double *X_out, bool out_dev, di_stats *st) {
    cudaStream_t s = g->stream;
    if (!g->X) {  // the in-link side and the iterates, at the first power iteration
        di_status r = build_transpose(g);
        if (r == DI_OK) r = power_alloc(g);
        if (r != DI_OK) return r;
    }
    if (!g->exec[2]) {
        di_status r = build_power_graph(g);
        if (r != DI_OK) return r;
    }
    PullArgs a = make_args(g);
    const int nparts = g->pull_blocks[0] + g->pull_blocks[1] + g->pull_blocks[2];
    DI_CUDA(cudaEventRecord(g->ev0, s));
    const int grid = std::max(1, std::min(g->num_sms * 8, (g->n + 255) / 256));
    k_power_init<<<grid, 256, 0, s>>>(a, tol, max_iter);
    DI_CUDA(cudaGetLastError());
    g->pprof_ms[0] = g->pprof_ms[1] = 0.0;
    if (profile) {
        // the graph body's two kernels launched from the host with events around each
        cudaGraphConditionalHandle none = 0;
        for (;;) {
            DI_CUDA(cudaEventRecord(g->pev[0], s));
            k_pull<<<nparts, 256, 0, s>>>(a);
            DI_CUDA(cudaEventRecord(g->pev[1], s));
            k_power_finalize<<<1, 256, 0, s>>>(a, nparts, none, 0);
            DI_CUDA(cudaEventRecord(g->pev[2], s));
            DI_CUDA(cudaGetLastError());
            DI_CUDA(cudaMemcpyAsync(g->h_pst, g->pst, sizeof(PowerState), cudaMemcpyDeviceToHost, s));
            DI_CUDA(cudaStreamSynchronize(s));
            float t0 = 0.f, t1 = 0.f;
            DI_CUDA(cudaEventElapsedTime(&t0, g->pev[0], g->pev[1]));
            DI_CUDA(cudaEventElapsedTime(&t1, g->pev[1], g->pev[2]));
            g->pprof_ms[0] += t0;
            g->pprof_ms[1] += t1;
            if (g->h_pst->done) break;
        }
    } else {
        DI_CUDA(cudaGraphLaunch(g->exec[2], s));
    }
    DI_CUDA(cudaEventRecord(g->ev1, s));
    DI_CUDA(cudaMemcpyAsync(g->h_pst, g->pst, sizeof(PowerState), cudaMemcpyDeviceToHost, s));
    if (X_out) {
        di_status r = gather_x(g, g->X, X_out, out_dev);
        if (r != DI_OK) return r;
    }
    DI_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    DI_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    const PowerState &h = *g->h_pst;
    if (st) {
        st->bound = h.delta * g->d / (1.0 - g->d);
        st->l1_F = h.delta;
        st->R = h.delta;
        st->edges_pushed = (int64_t)h.iters * g->nnz;
        st->sources_pushed = (int64_t)h.iters * g->n;
        st->sweeps = h.iters;
        st->converged = h.done == 1 ? 1 : 0;
        st->seconds = ms * 1e-3;
        st->kernel_launches = 1 + 2LL * h.iters;  // init + (pull, finalize) per product
    }
    if (h.done == 3) return set_error(DI_EKERNEL, "power iteration became non-finite");
    if (h.done != 1) return set_error(DI_ENOTCONVERGED, "power iteration hit max_iter before the stop rule");
    return DI_OK;
}

}  // namespace diter
