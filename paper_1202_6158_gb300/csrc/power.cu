// power.cu -- MAT-ITER, the plain comparison (Section 4): X_0 = 0,
// X_{k+1} = dPX_k + (1-d)V on the uncompleted P, stopped when
// |X_{k+1} - X_k|_1 * d/(1-d) < tol.
//
// Each product is a pull ("collection", Section 1) over the in-link lists:
//   y_j = (1-d)V_j + sum_{i -> j} z_i,   z_i = d * x_i / outdeg(i)  (0 if dangling)
// with z of the current iterate kept in one of two buffers so the gather never
// sees a value of the product being formed.  Three kernels per product:
//   k_pgather     the in-links, in target order, cut into even ranges: each lane takes
//                 kPowRun (32) consecutive links, gathers z of their sources (32 random
//                 8-byte loads in flight per lane hide the DRAM latency), sums them
//                 serially per target (one FP64 add per link) and adds each target's sum
//                 to the accumulator Y with one red.add;
//   k_pepilogue   streams the nodes: |y - x|, x = y, z = d*y/outdeg, Y = (1-d)V for the
//                 next product, with per-CTA sums of |y - x|;
//   k_power_finalize  one CTA reduces |X_{k+1} - X_k|_1 in fixed order and drives the
//                 CUDA-graph while-loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace diter {
namespace {

constexpr int kPowRun = 32;  // consecutive in-links per lane and step of the gather (gathers in flight)

__device__ double block_sum_d(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
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
    long long nnz;
    const int *in_src, *in_dst;
    const double *inv_deg;  // d / outdeg, 0 for dangling nodes
    const double *V;        // NULL: uniform
    double omd, d, u, omdu;
    double *X, *Z0, *Z1, *Y;
    PowerPartial *pp;
    PowerState *pst;
};

// (1-d) V_j
__device__ __forceinline__ double omdv_of(const PullArgs &a, int j) { return a.V ? a.omd * a.V[j] : a.omdu; }

__global__ void __launch_bounds__(256, 2) k_pgather(PullArgs a) {
    if (a.pst->done) return;
    const double *__restrict__ zc = a.pst->cur ? a.Z1 : a.Z0;
    constexpr int kStepLinks = 32 * kPowRun;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * 8, gw = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    // ranges of whole steps, so that every full run starts on a 32-byte boundary
    const long long per = (a.nnz + nwarps - 1) / nwarps + kStepLinks - 1;
    const long long span = per - per % kStepLinks;
    const long long e_beg = min(a.nnz, gw * span), e_end = min(a.nnz, e_beg + span);
    for (long long e0 = e_beg; e0 < e_end; e0 += kStepLinks) {
        const long long eb = e0 + (long long)kPowRun * lane;
        int src[kPowRun], dst[kPowRun];
        if (eb + kPowRun <= e_end) {
            const int4 *ps = reinterpret_cast<const int4 *>(a.in_src + eb);
            const int4 *pd = reinterpret_cast<const int4 *>(a.in_dst + eb);
#pragma unroll
            for (int h = 0; h < kPowRun / 4; ++h) {
                const int4 x = __ldg(ps + h), y = __ldg(pd + h);
                src[4 * h] = x.x; src[4 * h + 1] = x.y; src[4 * h + 2] = x.z; src[4 * h + 3] = x.w;
                dst[4 * h] = y.x; dst[4 * h + 1] = y.y; dst[4 * h + 2] = y.z; dst[4 * h + 3] = y.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kPowRun; ++k) {
                const bool in = eb + k < e_end;
                src[k] = in ? __ldg(a.in_src + eb + k) : -1;
                dst[k] = in ? __ldg(a.in_dst + eb + k) : -1;
            }
        }
        double v[kPowRun];
#pragma unroll
        for (int k = 0; k < kPowRun; ++k) v[k] = src[k] >= 0 ? zc[src[k]] : 0.0;
        int cur = dst[0];
        double acc = v[0];
#pragma unroll
        for (int k = 1; k < kPowRun; ++k) {
            if (dst[k] != cur) {
                if (cur >= 0 && acc != 0.0) red_add(a.Y + cur, acc);
                cur = dst[k];
                acc = 0.0;
            }
            acc += v[k];
        }
        if (cur >= 0 && acc != 0.0) red_add(a.Y + cur, acc);
    }
}

__global__ void __launch_bounds__(256) k_pepilogue(PullArgs a) {
    __shared__ double sh[8];
    if (a.pst->done) return;
    double *__restrict__ zn = a.pst->cur ? a.Z0 : a.Z1;
    double delta = 0.0;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (long long)gridDim.x * blockDim.x) {
        const double y = a.Y[j];
        delta += fabs(y - a.X[j]);
        a.X[j] = y;
        zn[j] = y * a.inv_deg[j];
        a.Y[j] = omdv_of(a, (int)j);  // the next product starts from (1-d)V
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
    double parts = 0.0;
    for (int c = threadIdx.x; c < nparts; c += blockDim.x) parts += a.pp[c].delta;
    parts = block_sum_d(parts, sh);
    if (threadIdx.x != 0) return;
    PowerState *p = a.pst;
    p->delta = parts;
    p->iters += 1;
    p->cur ^= 1;
    int done = 0;
    if (!isfinite(parts)) done = 3;
    else if (parts * p->d / (1.0 - p->d) < p->tol) done = 1;
    else if (p->iters >= p->max_iters) done = 2;
    p->done = done;
    if (done && in_graph) cudaGraphSetConditional(handle, 0);
}

__global__ void k_power_init(PullArgs a, double tol, int max_iters) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        a.X[i] = 0.0;
        a.Z0[i] = 0.0;
        a.Z1[i] = 0.0;
        a.Y[i] = omdv_of(a, (int)i);
    }
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
    a.nnz = g->nnz;
    a.in_src = g->in_src;
    a.in_dst = g->in_dst;
    a.inv_deg = g->inv_deg;
    a.V = g->V;
    a.omd = 1.0 - g->d;
    a.d = g->d;
    a.u = 1.0 / (double)g->n;
    a.omdu = a.omd * a.u;
    a.X = g->X;
    a.Z0 = g->Z[0];
    a.Z1 = g->Z[1];
    a.Y = g->Y;
    a.pp = g->ppart;
    a.pst = g->pst;
    return a;
}

int gather_grid(const di_graph *g) { return g->num_sms * 2; }  // one wave at 2 CTAs per SM
int epilogue_grid(const di_graph *g) { return std::max(1, std::min(g->num_sms * 8, (g->n + 255) / 256)); }

void launch_product(di_graph *g, const PullArgs &a, cudaStream_t s) {
    k_pgather<<<gather_grid(g), 256, 0, s>>>(a);
    k_pepilogue<<<epilogue_grid(g), 256, 0, s>>>(a);
}

di_status build_power_graph(di_graph *g) {
    PullArgs a = make_args(g);
    const int nparts = epilogue_grid(g);
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
    launch_product(g, a, g->cap);
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
    const int nparts = epilogue_grid(g);
    DI_CUDA(cudaMallocAsync(&g->X, sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->Z[0], sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->Z[1], sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->Y, sizeof(double) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&g->ppart, sizeof(PowerPartial) * (size_t)nparts, s));
    DI_CUDA(cudaMallocAsync(&g->pst, sizeof(PowerState), s));
    DI_CUDA(cudaMemsetAsync(g->pst, 0, sizeof(PowerState), s));
    return DI_OK;
}

di_status run_power(di_graph *g, double tol, int max_iter, int profile, double *X_out, bool out_dev, di_stats *st) {
    cudaStream_t s = g->stream;
    if (!g->X) {  // the in-link side and the iterates, at the first power iteration
        di_status r = build_in_dst(g);
        if (r == DI_OK) r = power_alloc(g);
        if (r != DI_OK) return r;
    }
    if (!g->exec[2]) {
        di_status r = build_power_graph(g);
        if (r != DI_OK) return r;
    }
    PullArgs a = make_args(g);
    const int nparts = epilogue_grid(g);
    DI_CUDA(cudaEventRecord(g->ev0, s));
    const int grid = std::max(1, std::min(g->num_sms * 8, (g->n + 255) / 256));
    k_power_init<<<grid, 256, 0, s>>>(a, tol, max_iter);
    DI_CUDA(cudaGetLastError());
    g->pprof_ms[0] = g->pprof_ms[1] = 0.0;
    if (profile) {
        // the graph body's kernels launched from the host with events around the product
        // (gather and epilogue) and the finalize
        cudaGraphConditionalHandle none = 0;
        for (;;) {
            DI_CUDA(cudaEventRecord(g->pev[0], s));
            launch_product(g, a, s);
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
        st->kernel_launches = 1 + 3LL * h.iters;  // init + (gather, epilogue, finalize) per product
    }
    if (h.done == 3) return set_error(DI_EKERNEL, "power iteration became non-finite");
    if (h.done != 1) return set_error(DI_ENOTCONVERGED, "power iteration hit max_iter before the stop rule");
    return DI_OK;
}

}  // namespace diter
