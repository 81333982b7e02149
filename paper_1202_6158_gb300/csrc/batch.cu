// batch.cu -- up to 64 personalized queries diffused together.
//
// Each query q has its own personalization vector V_q (its seed distribution;
// Section 2.1: V is the personalization vector), its own fluid F_q, history H_q
// and residual R_q.  The fluids are interleaved: row i of Fb holds F_q[i] for the
// K lanes q (K = 4, 8, 16, 32 or 64; FP32, 4K bytes), so one read of node i's
// out-links serves every query.  One sweep:
//
//   k_bscan    streams Fb (K/4 lanes per node row, one float4 of 4 queries per
//              lane).  Node i is selected when F_q[i] > T_q for some query q that
//              has not converged; its whole row is then exchanged -- every lane's
//              fluid moves -- which is a diffusion of node i for every query (any
//              choice of nodes is a valid sequence, Section 2.2).  The selected
//              (i, row) pairs go to the class lists of the single-query path,
//              through the same per-warp offsets; per-query |F|_1 and removed
//              mass are summed per lane and added to per-query accumulators.
//   k_bpush    adds the row to H_i (FP64) and, unless i is dangling, adds
//              row * d/outdeg(i) to the row of every child with one
//              red.global.add.v4.f32 per lane (4K bytes per out-link); the
//              hottest targets' rows are summed in shared memory first.  A
//              node's out-links are spread over a lane group (up to 8), a warp
//              (up to 1024) or the whole CTA, as in the single-query push.
//   k_bfinalize  one thread per query: R_q = |F_q|_1 - removed_q, T_q = beta R_q/n,
//              a query stops when R_q <= tol (1-d); the while-loop ends when all
//              have stopped.
//
// Then |F_q|_1 is recomputed in FP64 per query to confirm each stop, as for a
// single solve.  The loop is one CUDA graph (while-conditional node).  The rows
// are K floats apart for a fresh batch; a serving pool keeps its rows 4*cap_lanes
// bytes apart and runs the narrowest loop that covers its busy lanes.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace diter {
namespace {

constexpr int kBScanDepth = 4;  // steps of fluid rows each warp of the batched scan keeps in flight

__device__ __forceinline__ void red_add_v4(float *p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
}

__global__ void k_binit(long long rows, int n, int K, float *__restrict__ Fb, double *__restrict__ Hb) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < rows * K;
         t += (long long)gridDim.x * blockDim.x) {
        Fb[t] = 0.f;
        if (t < (long long)n * K) Hb[t] = 0.0;
    }
}

// F_q = (1-d) w_s / sum(w) on the seeds of query q
__global__ void k_bseeds(int nitems, int K, const int *__restrict__ q_of, const int *__restrict__ seeds,
                         const double *__restrict__ val, const int *__restrict__ new_of, float *__restrict__ Fb) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nitems; t += gridDim.x * blockDim.x)
        atomicAdd(&Fb[(long long)new_of[seeds[t]] * K + q_of[t]], (float)val[t]);
}

__global__ void k_bctl_init(int k, BatchQ *__restrict__ bq, BatchCtl *__restrict__ ctl, double tol, double omd,
                            double beta, int n, int max_sweeps) {
    const int q = threadIdx.x;
    if (q < kLanes) {
        BatchQ b;
        b.R = omd;
        b.tolR = tol * omd;
        b.l1_acc = 0.0;
        b.rem_acc = 0.0;
        b.l1_exact = 0.0;
        b.active = q < k ? 1 : 0;
        b.done = q < k ? (omd <= b.tolR ? 1 : 0) : 1;
        b.T = b.done ? INFINITY : beta * omd / (double)n;
        b.selected = 0;
        b.sweeps = 0;
        b.confirmed = 0;
        bq[q] = b;
    }
    if (q == 0) {
        ctl->sweeps = 0;
        ctl->max_sweeps = max_sweeps;
        ctl->edges = 0;
        ctl->srcs = 0;
        ctl->sel_edges = 0;
        ctl->pull = 0;
        ctl->beta = beta;
        ctl->body_runs = 0;
        ctl->round_sweeps = 0;
        ctl->round_cap = max_sweeps;
        ctl->stop_on_done = 0;
        ctl->lane_max_sweeps = INT_MAX;
        ctl->newly = 0;
        int all = 1;
        for (int i = 0; i < k; ++i) all &= (omd <= tol * omd) ? 1 : 0;
        ctl->all_done = all;
    }
}

// LPN lanes per node row (K = 4 LPN queries, a float4 per lane); 32/LPN rows per warp step
template <int LPN>
__global__ void __launch_bounds__(kScanThreads) k_bscan(int wchunk, int S, float *__restrict__ Fb,
                                                        const unsigned char *__restrict__ cls,
                                                        const int *__restrict__ region, int W,
                                                        int *__restrict__ fcount, int *__restrict__ pre,
                                                        unsigned *__restrict__ ticket, int *__restrict__ sel_node,
                                                        float *__restrict__ sel_rows, int *__restrict__ spos,
                                                        BatchQ *__restrict__ bq, BatchCtl *__restrict__ ctl, double d) {
    constexpr int K = 4 * LPN, NPS = 32 / LPN;
    __shared__ double s_l1[K], s_rem[K];
    __shared__ int s_sel[K];
    __shared__ unsigned s_ticket;
    if (ctl->all_done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, h = lane / LPN, lq = lane % LPN;
    const unsigned gmask = ((LPN == 32 ? 0xffffffffu : ((1u << LPN) - 1u))) << (h * LPN);
    const unsigned lt = (1u << lane) - 1u;
    if (threadIdx.x < K) {
        s_l1[threadIdx.x] = 0.0;
        s_rem[threadIdx.x] = 0.0;
        s_sel[threadIdx.x] = 0;
    }
    __syncthreads();
    float T4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) T4[k] = (float)bq[4 * lq + k].T;  // +inf for queries that stopped
    const float omd = (float)(1.0 - d);
    const int g = blockIdx.x * kWarps + w;
    const long long wbeg = (long long)g * wchunk;
    int run[kLists], start[kLists];
#pragma unroll
    for (int L = 0; L < kLists; ++L) start[L] = run[L] = region[L * (W + 1) + g];
    float l1[4] = {0.f, 0.f, 0.f, 0.f}, rem[4] = {0.f, 0.f, 0.f, 0.f};
    int sel4[4] = {0, 0, 0, 0};
    int nsel = 0;
    int hub_chunks = 0;  // chunks of the hub rows this lane listed (group leaders only)
    const bool pull = ctl->pull != 0;  // the push kernel reads the lists, the pull kernel the positions
    const int nsteps = wchunk / NPS;
    // kBScanDepth steps of rows in flight per warp (a register ring, unrolled so it stays in registers)
    float4 buf[kBScanDepth];
    int cb[kBScanDepth];
#pragma unroll
    for (int d = 0; d < kBScanDepth; ++d) {
        buf[d] = make_float4(0.f, 0.f, 0.f, 0.f);
        cb[d] = 0;
        if (d < nsteps) {
            buf[d] = *reinterpret_cast<const float4 *>(Fb + (wbeg + (long long)NPS * d + h) * S + 4 * lq);
            cb[d] = cls[wbeg + (long long)NPS * d + h];
        }
    }
    // nsteps is a multiple of kBScanDepth: a warp's sub-chunk is a multiple of kStep (256) nodes
    // and a step covers NPS <= 32 of them
    static_assert((kStep / 32) % kBScanDepth == 0, "whole rounds of the register ring per sub-chunk");
    for (int s0 = 0; s0 < nsteps; s0 += kBScanDepth) {
#pragma unroll
        for (int dd = 0; dd < kBScanDepth; ++dd) {
            const int s = s0 + dd;
            const long long node = wbeg + (long long)NPS * s + h;
            const float4 cur = buf[dd];
            const int cbyte = cb[dd];               // class byte: 2 + chunks for a hub row
            const int ccur = class_of_byte(cbyte);
            if (s + kBScanDepth < nsteps) {
                buf[dd] = *reinterpret_cast<const float4 *>(Fb + (node + (long long)NPS * kBScanDepth) * S + 4 * lq);
                cb[dd] = cls[node + (long long)NPS * kBScanDepth];
            }
            const float v[4] = {cur.x, cur.y, cur.z, cur.w};
            bool above = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                l1[k] += v[k];
                const bool a = v[k] > T4[k];
                above |= a;
                sel4[k] += a ? 1 : 0;
            }
            const unsigned bal = __ballot_sync(kFull, above);
            const bool act = (bal & gmask) != 0;
            // ordered positions: one bit per group leader for each class
            const bool leader = lq == 0;
            int pos = 0;
#pragma unroll
            for (int L = 0; L < kLists; ++L) {
                const unsigned bits = __ballot_sync(kFull, leader && act && ccur == L);
                if (ccur == L) pos = run[L] + __popc(bits & lt & ~gmask & ((1u << (h * LPN)) - 1u));
                run[L] += __popc(bits);
            }
            if (leader && act && ccur == 3) hub_chunks += cbyte - 2;
            if (act) {
                const float f = ccur == 0 ? 1.f : omd;  // a dangling node's fluid leaves entirely (Section 3.3)
#pragma unroll
                for (int k = 0; k < 4; ++k) rem[k] += f * v[k];
                *reinterpret_cast<float4 *>(sel_rows + (long long)pos * K + 4 * lq) = cur;
                if (lq == 0) {
                    sel_node[pos] = (int)node;
                    nsel += 1;
                }
                *reinterpret_cast<float4 *>(Fb + node * S + 4 * lq) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (pull && lq == 0) spos[node] = act ? pos : -1;
        }
    }
    hub_chunks = __reduce_add_sync(kFull, hub_chunks);
    if (lane == 0) {
#pragma unroll
        for (int L = 0; L < kLists; ++L) fcount[L * W + g] = run[L] - start[L];
        fcount[kChunkRow * W + g] = hub_chunks;
    }
    // per-query sums: the groups of a warp, then the CTA, then one atomic per query
#pragma unroll
    for (int o = LPN; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            l1[k] += __shfl_xor_sync(kFull, l1[k], o);
            rem[k] += __shfl_xor_sync(kFull, rem[k], o);
            sel4[k] += __shfl_xor_sync(kFull, sel4[k], o);
        }
    }
    if (h == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(&s_l1[4 * lq + k], (double)l1[k]);
            atomicAdd(&s_rem[4 * lq + k], (double)rem[k]);
            atomicAdd(&s_sel[4 * lq + k], sel4[k]);
        }
    }
    __syncthreads();
    if (lq == 0 && nsel) atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->srcs), (unsigned long long)nsel);
    if (threadIdx.x < K && bq[threadIdx.x].active) {
        atomicAdd(&bq[threadIdx.x].l1_acc, s_l1[threadIdx.x]);
        atomicAdd(&bq[threadIdx.x].rem_acc, s_rem[threadIdx.x]);
        if (s_sel[threadIdx.x]) atomicAdd(&bq[threadIdx.x].selected, s_sel[threadIdx.x]);
    }
    // the last CTA turns the per-warp counts into prefix sums for the push
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1u);
    __syncthreads();
    if (s_ticket == gridDim.x - 1) {
        __threadfence();
        prefix_counts(fcount, W, pre);
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// one out-link j of a selected node: this lane's 4 queries of row j += wv
template <int K>
__device__ __forceinline__ void bpush_edge(float *__restrict__ Fb, int S, float *hot, int n_hot, int j, int l16,
                                           float4 wv) {
    if (j < n_hot) {
        float *hp = hot + j * K + 4 * l16;
        atomicAdd(hp, wv.x);
        atomicAdd(hp + 1, wv.y);
        atomicAdd(hp + 2, wv.z);
        atomicAdd(hp + 3, wv.w);
    } else {
        red_add_v4(Fb + (long long)j * S + 4 * l16, wv);
    }
}

// H_i += row for the 4 queries of this lane (FP64; node i is pushed by one lane group only)
__device__ __forceinline__ void bpush_h(double *__restrict__ Hb, int S, int node, int l16, const float4 row) {
    double2 *hp = reinterpret_cast<double2 *>(Hb + (long long)node * S + 4 * l16);
    double2 a = hp[0], b = hp[1];
    a.x += row.x;
    a.y += row.y;
    b.x += row.z;
    b.y += row.w;
    hp[0] = a;
    hp[1] = b;
}

// row * d/outdeg to every child of a row {beg, deg}; this lane group takes out-links
// e_beg, e_beg + e_step, ...
template <int K>
__device__ __forceinline__ void bpush_row(int beg, int deg, float inv, const float4 row, int l16,
                                          const int *__restrict__ col_idx, float *__restrict__ Fb, int S, float *hot,
                                          int n_hot, int e_beg, int e_step) {
    const float4 wv = make_float4(row.x * inv, row.y * inv, row.z * inv, row.w * inv);
    int e = e_beg;
    for (; e + 3 * e_step < deg; e += 4 * e_step) {
        const int j0 = __ldg(col_idx + beg + e), j1 = __ldg(col_idx + beg + e + e_step);
        const int j2 = __ldg(col_idx + beg + e + 2 * e_step), j3 = __ldg(col_idx + beg + e + 3 * e_step);
        bpush_edge<K>(Fb, S, hot, n_hot, j0, l16, wv);
        bpush_edge<K>(Fb, S, hot, n_hot, j1, l16, wv);
        bpush_edge<K>(Fb, S, hot, n_hot, j2, l16, wv);
        bpush_edge<K>(Fb, S, hot, n_hot, j3, l16, wv);
    }
    for (; e < deg; e += e_step) bpush_edge<K>(Fb, S, hot, n_hot, __ldg(col_idx + beg + e), l16, wv);
}

template <int LPN>
__global__ void __launch_bounds__(kScanThreads, 4) k_bpush(const RowRec<float> *__restrict__ rec,
                                                        const int *__restrict__ col_idx, float *__restrict__ Fb,
                                                        double *__restrict__ Hb, int S, const int *__restrict__ region,
                                                        const int *__restrict__ pre,
                                                        const int *__restrict__ fcount, int W,
                                                        const int *__restrict__ sel_node,
                                                        const float *__restrict__ sel_rows, int n_hot,
                                                        BatchCtl *__restrict__ ctl) {
    constexpr int K = 4 * LPN, GPC = kScanThreads / LPN;   // lane groups per CTA
    __shared__ float hot[kBatchHot * K];
    __shared__ long long s_red[kWarps];
    if (ctl->all_done || ctl->pull) return;
    for (int t = threadIdx.x; t < kBatchHot * K; t += kScanThreads) hot[t] = 0.f;
    __syncthreads();
    const int grp = threadIdx.x / LPN, lq = threadIdx.x % LPN;
    const int ngrp = gridDim.x * GPC, ggrp = blockIdx.x * GPC + grp;
    long long edges = 0;  // out-links of the pushed nodes
    // class 3: the hub rows, cut into chunks of at most kHubChunk out-links; CTA b takes the
    // contiguous chunk range [b nch / grid, (b+1) nch / grid), each lane group taking every GPC-th
    // out-link of a chunk.  The chunks are numbered sub-chunk by sub-chunk through the prefix sums
    // of the scan's per-warp chunk counts, then entry by entry; a row's first chunk also adds its
    // fluid row to H.
    {
        const int *pch = pre + kChunkRow * (W + 1), *r3 = region + 3 * (W + 1), *f3 = fcount + 3 * W;
        const int nch = __ldg(pch + W);
        const int c0 = (int)((long long)blockIdx.x * nch / gridDim.x);
        const int c1 = (int)((long long)(blockIdx.x + 1) * nch / gridDim.x);
        if (c0 < c1) {
            // the walk's state is the same in every thread (broadcast loads)
            int gs = find_sub(pch, W, c0);
            int e = __ldg(r3 + gs), e_end = e + __ldcg(f3 + gs), cum = __ldg(pch + gs);
            int node = sel_node[e];
            RowRec<float> rr = rec[node];
            int nc = hub_chunk_count(rr.deg);
            for (int c = c0; c < c1; ++c) {
                while (c >= cum + nc) {
                    cum += nc;
                    if (++e >= e_end) {
                        do {
                            ++gs;
                        } while (__ldcg(f3 + gs) == 0);
                        e = __ldg(r3 + gs);
                        e_end = e + __ldcg(f3 + gs);
                    }
                    node = sel_node[e];
                    rr = rec[node];
                    nc = hub_chunk_count(rr.deg);
                }
                const int clen = hub_chunk_len(rr.deg, nc), j = c - cum;
                const int off = j * clen, len = min(clen, rr.deg - off);
                const float4 row = *reinterpret_cast<const float4 *>(sel_rows + (long long)e * K + 4 * lq);
                if (grp == 0) {
                    if (j == 0) bpush_h(Hb, S, node, lq, row);  // H once per row
                    if (lq == 0) edges += len;
                }
                bpush_row<K>(rr.beg + off, len, rr.inv, row, lq, col_idx, Fb, S, hot, n_hot, grp, GPC);
            }
        }
    }
    // class 2: a warp per node, its 32/LPN lane groups taking every (32/LPN)-th out-link.  The
    // ranks are strided over the warps (rank t to warp t mod nwarps); lane j first finds and
    // loads the list position, node and row record of the warp's j-th node of each group of 32
    {
        constexpr int GPW = 32 / LPN;
        const int lane = threadIdx.x & 31, gi = lane / LPN;
        const int nwarps = gridDim.x * kWarps, gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
        const int *p2 = pre + 2 * (W + 1), *r2 = region + 2 * (W + 1);
        const int tot = __ldg(p2 + W);
        for (long long k0 = 0; gw + k0 * nwarps < tot; k0 += 32) {
            const long long t = gw + (k0 + lane) * nwarps;
            int mpos = 0, mnode = 0, mb = 0, md = 0;
            float mi = 0.f;
            if (t < tot) {
                const int gs = find_sub(p2, W, (int)t);
                mpos = __ldg(r2 + gs) + ((int)t - __ldg(p2 + gs));
                mnode = sel_node[mpos];
                const RowRec<float> rr = rec[mnode];
                mb = rr.beg;
                md = rr.deg;
                mi = rr.inv;
            }
            const int m = (int)min(32LL, (tot - gw - k0 * nwarps + nwarps - 1) / nwarps);
            for (int j = 0; j < m; ++j) {
                const int pos = __shfl_sync(kFull, mpos, j), node = __shfl_sync(kFull, mnode, j);
                const int rb = __shfl_sync(kFull, mb, j), rd = __shfl_sync(kFull, md, j);
                const float ri = __shfl_sync(kFull, mi, j);
                const float4 row = *reinterpret_cast<const float4 *>(sel_rows + (long long)pos * K + 4 * lq);
                if (gi == 0) {
                    bpush_h(Hb, S, node, lq, row);
                    if (lq == 0) edges += rd;
                }
                bpush_row<K>(rb, rd, ri, row, lq, col_idx, Fb, S, hot, n_hot, gi, GPW);
            }
        }
    }
    // classes 0, 1: a lane group per node, contiguous rank ranges per group; lane q of a
    // group first finds and loads the position, node and row record of the group's q-th
    // node of each run of LPN
    {
        const int lane = threadIdx.x & 31;
        const unsigned gmask = (LPN == 32 ? kFull : ((1u << LPN) - 1u)) << (lane & ~(LPN - 1));
        for (int L = 0; L < 2; ++L) {
            const int *pl = pre + L * (W + 1), *rl = region + L * (W + 1);
            const int tot = __ldg(pl + W);
            const int per = (tot + ngrp - 1) / ngrp;
            const int t_beg = min(tot, ggrp * per), t_end = min(tot, t_beg + per);
            int gl = 0;
            if (t_beg < t_end) gl = find_sub(pl, W, t_beg);   // the same in every lane of the group
            for (int i0 = 0; i0 < per; i0 += LPN) {
                const int t = t_beg + i0 + lq;
                int mpos = 0, mnode = 0, mb = 0, md = 0, mg = gl;
                float mi = 0.f;
                if (t < t_end) {
                    mg = find_sub_from(pl, W, t, gl);
                    mpos = __ldg(rl + mg) + (t - __ldg(pl + mg));
                    mnode = sel_node[mpos];
                    if (L == 1) {
                        const RowRec<float> rr = rec[mnode];
                        mb = rr.beg;
                        md = rr.deg;
                        mi = rr.inv;
                    }
                }
#pragma unroll
                for (int o = 1; o < LPN; o <<= 1) mg = max(mg, __shfl_xor_sync(gmask, mg, o, LPN));
                gl = mg;
                const int m = min(LPN, t_end - (t_beg + i0));
                for (int j = 0; j < m; ++j) {
                    const int pos = __shfl_sync(gmask, mpos, j, LPN), node = __shfl_sync(gmask, mnode, j, LPN);
                    const float4 row = *reinterpret_cast<const float4 *>(sel_rows + (long long)pos * K + 4 * lq);
                    bpush_h(Hb, S, node, lq, row);
                    if (L == 1) {
                        const int rb = __shfl_sync(gmask, mb, j, LPN), rd = __shfl_sync(gmask, md, j, LPN);
                        const float ri = __shfl_sync(gmask, mi, j, LPN);
                        if (lq == 0) edges += rd;
                        bpush_row<K>(rb, rd, ri, row, lq, col_idx, Fb, S, hot, n_hot, 0, 1);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_hot * K; t += kScanThreads) {
        const float v = hot[t];
        if (v != 0.f) atomicAdd(Fb + (long long)(t / K) * S + t % K, v);
    }
    const long long be = block_sum(edges, s_red);
    if (threadIdx.x == 0 && be)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->sel_edges), (unsigned long long)be);
}

__device__ __forceinline__ bool nonzero4(const float4 r) { return r.x != 0.f || r.y != 0.f || r.z != 0.f || r.w != 0.f; }

__device__ __forceinline__ void fma4(float4 &acc, const float4 r, float w) {
    acc.x = fmaf(r.x, w, acc.x);
    acc.y = fmaf(r.y, w, acc.y);
    acc.z = fmaf(r.z, w, acc.z);
    acc.w = fmaf(r.w, w, acc.w);
}

// The pull direction of a dense sweep: the same diffusion as k_bpush, read from the target
// side.  First every selected node's row goes to H (contiguous rank ranges per lane group).
// Then the in-links, in target order, are cut into even ranges, one per lane group: the
// group walks its range, gathers row(src) * d/outdeg(src) of every selected source from the
// compact list of the sweep (small enough to stay in L2), sums the in-links of one target
// in registers and adds the sum to the target's row with one red.global.add.v4.f32 per lane
// (an atomic only because a target's in-links may straddle two ranges).
template <int LPN>
__global__ void __launch_bounds__(kScanThreads, 4) k_bpull(const RowRec<float> *__restrict__ rec,
                                                        const int *__restrict__ in_src,
                                                        const int *__restrict__ in_dst,
                                                        const float *__restrict__ inv_deg, long long nnz,
                                                        const int *__restrict__ spos, float *__restrict__ Fb,
                                                        double *__restrict__ Hb, int S, const int *__restrict__ region,
                                                        const int *__restrict__ pre, int W,
                                                        const int *__restrict__ sel_node,
                                                        const float *__restrict__ sel_rows,
                                                        BatchCtl *__restrict__ ctl) {
    constexpr int K = 4 * LPN, GPC = kScanThreads / LPN;
    __shared__ long long s_red[kWarps];
    if (ctl->all_done || !ctl->pull) return;
    const int lane = threadIdx.x & 31, grp = threadIdx.x / LPN, lq = threadIdx.x % LPN;
    const int ngrp = gridDim.x * GPC, ggrp = blockIdx.x * GPC + grp;
    const unsigned gmask = (LPN == 32 ? kFull : ((1u << LPN) - 1u)) << (lane & ~(LPN - 1));
    // H_i += row_i for every selected node, all classes; their out-links are counted here
    long long edges = 0;
    for (int L = 0; L < kLists; ++L) {
        const int *pl = pre + L * (W + 1), *rl = region + L * (W + 1);
        const int tot = __ldg(pl + W);
        const int per = (tot + ngrp - 1) / ngrp;
        const int t_beg = min(tot, ggrp * per), t_end = min(tot, t_beg + per);
        int gl = 0;
        if (t_beg < t_end) gl = find_sub(pl, W, t_beg);
        for (int i0 = 0; i0 < per; i0 += LPN) {
            const int t = t_beg + i0 + lq;
            int mpos = 0, mnode = 0, mg = gl;
            if (t < t_end) {
                mg = find_sub_from(pl, W, t, gl);
                mpos = __ldg(rl + mg) + (t - __ldg(pl + mg));
                mnode = sel_node[mpos];
                if (L > 0) edges += __ldg(&rec[mnode].deg);
            }
#pragma unroll
            for (int o = 1; o < LPN; o <<= 1) mg = max(mg, __shfl_xor_sync(gmask, mg, o, LPN));
            gl = mg;
            const int m = min(LPN, t_end - (t_beg + i0));
            for (int j = 0; j < m; ++j) {
                const int pos = __shfl_sync(gmask, mpos, j, LPN), node = __shfl_sync(gmask, mnode, j, LPN);
                bpush_h(Hb, S, node, lq, *reinterpret_cast<const float4 *>(sel_rows + (long long)pos * K + 4 * lq));
            }
        }
    }
    // the in-links
    constexpr int kU = 4;  // rows gathered before they are summed
    const long long per = (nnz + ngrp - 1) / ngrp;
    const long long e_beg = min(nnz, (long long)ggrp * per), e_end = min(nnz, e_beg + per);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int cur = -1;
    for (long long i0 = 0; i0 < per; i0 += LPN) {
        const long long e = e_beg + i0 + lq;
        int mdst = -1, mpos = -1;
        float mw = 0.f;
        if (e < e_end) {
            const int src = __ldg(in_src + e);
            mdst = __ldg(in_dst + e);
            mpos = __ldg(spos + src);
            mw = __ldg(inv_deg + src);
        }
        const int m = (int)min((long long)LPN, e_end - e_beg - i0);
        for (int j0 = 0; j0 < m; j0 += kU) {
            float4 r[kU];
            int dd[kU];
            float ww[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = (j0 + u) & (LPN - 1);
                const int pj = __shfl_sync(gmask, mpos, j, LPN);
                dd[u] = __shfl_sync(gmask, mdst, j, LPN);
                ww[u] = __shfl_sync(gmask, mw, j, LPN);
                r[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j0 + u < m && pj >= 0) r[u] = *reinterpret_cast<const float4 *>(sel_rows + (long long)pj * K + 4 * lq);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (j0 + u < m) {
                    if (dd[u] != cur) {
                        if (cur >= 0 && nonzero4(acc)) red_add_v4(Fb + (long long)cur * S + 4 * lq, acc);
                        acc = make_float4(0.f, 0.f, 0.f, 0.f);
                        cur = dd[u];
                    }
                    fma4(acc, r[u], ww[u]);
                }
            }
        }
    }
    if (cur >= 0 && nonzero4(acc)) red_add_v4(Fb + (long long)cur * S + 4 * lq, acc);
    const long long be = block_sum(edges, s_red);
    if (threadIdx.x == 0 && be)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->sel_edges), (unsigned long long)be);
}

// one thread per lane.  The loop ends when no lane is open or at the sweep limit; a
// serving round also ends after round_cap sweeps, or when a lane stops (stop_on_done).
__global__ void k_bfinalize(int n, long long pull_edges, BatchQ *__restrict__ bq, BatchCtl *__restrict__ ctl,
                            cudaGraphConditionalHandle handle, int in_graph) {
    __shared__ int s_open, s_newly;
    if (ctl->all_done) {
        if (threadIdx.x == 0) {
            ctl->body_runs += 1;
            if (in_graph) cudaGraphSetConditional(handle, 0);
        }
        return;
    }
    if (threadIdx.x == 0) {
        s_open = 0;
        s_newly = 0;
    }
    __syncthreads();
    const int q = threadIdx.x;
    if (q < kLanes) {
        BatchQ b = bq[q];
        if (b.active) {
            const double R = b.l1_acc - b.rem_acc;  // |F_q|_1 after the sweep
            const double Rprev = b.R;
            b.R = R > 0.0 ? R : 0.0;
            b.l1_acc = 0.0;
            b.rem_acc = 0.0;
            if (!b.done) {
                b.sweeps += 1;
                if (b.R <= b.tolR || b.sweeps >= ctl->lane_max_sweeps) {
                    b.done = b.R <= b.tolR ? 1 : 2;
                    b.T = INFINITY;
                    b.l1_exact = 0.0;  // summed by the confirmation that follows the loop
                    atomicAdd(&s_newly, 1);
                } else {
                    // T_q = beta R_q / n; halved when the query selected no node this sweep
                    b.T = (b.selected == 0 || !(b.R < Rprev)) ? 0.5 * b.T : ctl->beta * b.R / (double)n;
                    atomicAdd(&s_open, 1);
                }
            }
            b.selected = 0;
            bq[q] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the next sweep pulls when this one's selected nodes held at least pull_edges out-links
        const long long se = ctl->sel_edges;
        ctl->edges += se;
        ctl->sel_edges = 0;
        ctl->pull = se >= pull_edges ? 1 : 0;
        ctl->body_runs += 1;
        ctl->sweeps += 1;
        ctl->round_sweeps += 1;
        if (s_newly) ctl->newly = 1;
        if (s_open == 0)
            ctl->all_done = 1;
        else if (ctl->sweeps >= ctl->max_sweeps)
            ctl->all_done = 2;
        const bool stop = ctl->all_done != 0 || ctl->round_sweeps >= ctl->round_cap ||
                          (ctl->stop_on_done && s_newly != 0);
        if (stop && in_graph) cudaGraphSetConditional(handle, 0);
    }
}

// exact per-query |F_q|_1 in FP64 (a lane per query column, rows strided over the grid)
__global__ void k_bl1_exact(long long rows, int K, int S, const float *__restrict__ Fb, BatchQ *__restrict__ bq) {
    const int q = threadIdx.x % K;
    const int rstep = (gridDim.x * blockDim.x) / K;
    double a = 0.0;
    for (long long r = (long long)(blockIdx.x * blockDim.x + threadIdx.x) / K; r < rows; r += rstep)
        a += fabs((double)Fb[r * S + q]);
    atomicAdd(&bq[q].l1_exact, a);
}

__global__ void k_bzero_exact(BatchQ *__restrict__ bq) {
    if (threadIdx.x < kLanes) bq[threadIdx.x].l1_exact = 0.0;
}

// a stop the exact norm does not confirm re-opens that query
__global__ void k_bconfirm(int n, BatchQ *__restrict__ bq, BatchCtl *__restrict__ ctl) {
    __shared__ int s_open;
    if (threadIdx.x == 0) s_open = 0;
    __syncthreads();
    const int q = threadIdx.x;
    if (q < kLanes && bq[q].active && bq[q].done && !(bq[q].l1_exact <= bq[q].tolR)) {
        bq[q].done = 0;
        bq[q].R = bq[q].l1_exact;
        bq[q].T = ctl->beta * bq[q].l1_exact / (double)n;
        atomicAdd(&s_open, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_open && ctl->all_done == 1) ctl->all_done = 0;
}

// out[q][i] = Hb[new_of[i]][q] for the first k queries, back in the caller's numbering.  A
// CTA transposes a tile of kGatherTile nodes through shared memory: it reads their K-wide
// rows, then writes kGatherTile consecutive outputs of each query.
constexpr int kGatherTile = 32;
__global__ void __launch_bounds__(256) k_bgather(int n, int k, int K, const int *__restrict__ new_of,
                                                 const double *__restrict__ Hb, double *__restrict__ out) {
    __shared__ double tile[kGatherTile][kLanes + 1];
    const int ntiles = (n + kGatherTile - 1) / kGatherTile;
    for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const int i0 = b * kGatherTile;
        for (int t = threadIdx.x; t < kGatherTile * K; t += blockDim.x) {
            const int ii = t / K, q = t % K;
            if (i0 + ii < n && q < k) tile[ii][q] = Hb[(long long)new_of[i0 + ii] * K + q];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kGatherTile * k; t += blockDim.x) {
            const int q = t / kGatherTile, ii = t % kGatherTile;
            if (i0 + ii < n) out[(long long)q * n + i0 + ii] = tile[ii][q];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- serving rounds
//
// A serving loop keeps each lane busy with a stream of queries: between two launches
// of the captured loop, stopped lanes are copied out and cleared, and new queries
// start in the freed lanes while the others carry on where they were.

// frees and starts lanes, then opens the round
__global__ void k_bround_begin(LaneAdmin a, int n, double omd, double beta, int round_cap, int lane_max,
                               BatchQ *__restrict__ bq, BatchCtl *__restrict__ ctl) {
    __shared__ int s_open;
    if (threadIdx.x == 0) s_open = 0;
    __syncthreads();
    const int q = threadIdx.x;
    if (q < kLanes) {
        BatchQ b = bq[q];
        const unsigned long long bit = 1ull << q;
        if ((a.retire | a.admit) & bit) {
            b.R = 0.0;
            b.T = INFINITY;
            b.tolR = 0.0;
            b.l1_acc = 0.0;
            b.rem_acc = 0.0;
            b.l1_exact = 0.0;
            b.active = 0;
            b.done = 1;
            b.selected = 0;
            b.sweeps = 0;
            b.confirmed = 0;
        }
        if (a.admit & bit) {  // F_q = (1-d) V_q was added by the seeding kernel: R_q = 1-d
            b.active = 1;
            b.R = omd;
            b.tolR = a.tolR[q];
            b.done = omd <= b.tolR ? 1 : 0;
            b.T = b.done ? INFINITY : beta * omd / (double)n;
        }
        if (b.active && !b.done) atomicAdd(&s_open, 1);
        bq[q] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->round_sweeps = 0;
        ctl->round_cap = round_cap;
        ctl->stop_on_done = 1;
        ctl->lane_max_sweeps = lane_max;
        ctl->max_sweeps = INT_MAX;
        ctl->beta = beta;
        ctl->newly = 0;
        ctl->all_done = s_open ? 0 : 1;
    }
}

// exact FP64 |F_q|_1 of the lanes that stopped and are not confirmed yet; each thread
// keeps one lane and strides over the rows
__global__ void k_bl1_pending(long long rows, int K, const float *__restrict__ Fb, BatchQ *__restrict__ bq) {
    __shared__ int s_lane[kLanes];
    __shared__ double s_acc[kLanes];
    __shared__ int s_P;
    if (threadIdx.x == 0) {
        int P = 0;
        for (int q = 0; q < K; ++q)
            if (bq[q].active && bq[q].done && !bq[q].confirmed) s_lane[P++] = q;
        s_P = P;
    }
    if (threadIdx.x < kLanes) s_acc[threadIdx.x] = 0.0;
    __syncthreads();
    const int P = s_P;
    if (P == 0) return;
    const long long total = (long long)gridDim.x * blockDim.x;
    const long long Tp = (total / P) * P;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < Tp) {
        const int li = (int)(gid % P), q = s_lane[li];
        const long long rstep = Tp / P;
        double acc = 0.0;
        for (long long r = gid / P; r < rows; r += rstep) acc += fabs((double)Fb[r * K + q]);
        atomicAdd(&s_acc[li], acc);
    }
    __syncthreads();
    if (threadIdx.x < P) atomicAdd(&bq[s_lane[threadIdx.x]].l1_exact, s_acc[threadIdx.x]);
}

// a stop the exact norm does not confirm re-opens that lane; a lane at its sweep limit is
// confirmed as it stands (its bound is the exact norm)
__global__ void k_bconfirm_pending(int n, double beta, BatchQ *__restrict__ bq) {
    const int q = threadIdx.x;
    if (q >= kLanes) return;
    BatchQ b = bq[q];
    if (!(b.active && b.done && !b.confirmed)) return;
    b.R = b.l1_exact;
    if (b.done == 2 || b.l1_exact <= b.tolR) {
        b.confirmed = 1;
    } else {
        b.done = 0;
        b.T = beta * b.l1_exact / (double)n;
    }
    bq[q] = b;
}

// out_l[perm[r]] = Hb[r][lane_l]; the lane's history and fluid columns are cleared
__global__ void k_blane_retire(LaneRetire rl, int n, int K, const int *__restrict__ perm, double *__restrict__ Hb,
                               float *__restrict__ Fb) {
    const int cnt = rl.count;
    const long long total = (long long)n * cnt;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / cnt;
        const int li = (int)(t - r * cnt), q = rl.lane[li];
        const long long at = r * K + q;
        const double v = Hb[at];
        Hb[at] = 0.0;
        Fb[at] = 0.f;
        if (rl.out[li]) rl.out[li][perm[r]] = v;
    }
}

// one sweep of the batched loop on stream st: scan, push, pull, finalize.  In a capture the
// finalize drives the while-loop (in_graph = 1); a profiled loop passes four events, recorded
// before the scan, after it, after the push and pull, and after the finalize.
template <int LPN>
void launch_batch_sweep(di_graph *g, BatchPool *p, int S, cudaStream_t st, cudaGraphConditionalHandle handle,
                        int in_graph, cudaEvent_t *ev) {
    const int nhot = std::min(g->n_hot, kBatchHot);
    if (ev) cudaEventRecord(ev[0], st);
    k_bscan<LPN><<<g->G, kScanThreads, 0, st>>>(g->chunk / kWarps, S, p->Fb, g->cls, g->region, g->W, p->fcount,
                                                p->pre, p->ticket, p->selb_node, p->selb_rows, p->spos, p->bq,
                                                p->bctl, g->d);
    if (ev) cudaEventRecord(ev[1], st);
    // the width's settings (di_autotune_batch): push and pull grid, and the share of all
    // out-links that makes a sweep dense
    constexpr int slot = LPN == 1 ? 0 : (LPN == 2 ? 1 : (LPN == 4 ? 2 : (LPN == 8 ? 3 : 4)));
    const BatchTune &bt = g->btune[slot];
    const int grid = std::max(g->G, bt.push_per_sm * g->num_sms);
    k_bpush<LPN><<<grid, kScanThreads, 0, st>>>(g->rec32, g->col_idx, p->Fb, p->Hb, S, g->region, p->pre,
                                                p->fcount, g->W, p->selb_node, p->selb_rows, nhot, p->bctl);
    k_bpull<LPN><<<grid, kScanThreads, 0, st>>>(g->rec32, g->in_src, g->in_dst, g->inv_deg32, g->nnz, p->spos,
                                                p->Fb, p->Hb, S, g->region, p->pre, g->W, p->selb_node,
                                                p->selb_rows, p->bctl);
    if (ev) cudaEventRecord(ev[2], st);
    // rows of 4 lanes always push: their 16-byte reductions cost no more than the pull's gathers
    const long long share = std::max(1, bt.pull_share);
    const long long pull_edges = LPN >= 2 ? std::max(1LL, (g->nnz + share - 1) / share) : LLONG_MAX;
    k_bfinalize<<<1, kLanes, 0, st>>>(g->n, pull_edges, p->bq, p->bctl, handle, in_graph);
    if (ev) cudaEventRecord(ev[3], st);
}

template <int LPN>
void capture_batch_body(di_graph *g, BatchPool *p, cudaGraphConditionalHandle handle, int S) {
    launch_batch_sweep<LPN>(g, p, S, g->cap, handle, 1, nullptr);
}

// the batched loop launched from the host, sweep by sweep, with CUDA events around the kernels
di_status profile_batch_loop(di_graph *g, BatchPool *p, int slot, int S, cudaStream_t st, di_profile *prof) {
    cudaGraphConditionalHandle none = 0;
    int pulling = p->h_bctl->pull;  // the direction the next sweep takes
    for (int sw = 0; sw < (1 << 24); ++sw) {
        switch (slot) {
            case 0: launch_batch_sweep<1>(g, p, S, st, none, 0, g->pev); break;
            case 1: launch_batch_sweep<2>(g, p, S, st, none, 0, g->pev); break;
            case 2: launch_batch_sweep<4>(g, p, S, st, none, 0, g->pev); break;
            case 3: launch_batch_sweep<8>(g, p, S, st, none, 0, g->pev); break;
            default: launch_batch_sweep<16>(g, p, S, st, none, 0, g->pev); break;
        }
        DI_CUDA(cudaGetLastError());
        DI_CUDA(cudaMemcpyAsync(p->h_bctl, p->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
        DI_CUDA(cudaStreamSynchronize(st));
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        DI_CUDA(cudaEventElapsedTime(&t0, g->pev[0], g->pev[1]));
        DI_CUDA(cudaEventElapsedTime(&t1, g->pev[1], g->pev[2]));
        DI_CUDA(cudaEventElapsedTime(&t2, g->pev[2], g->pev[3]));
        prof->scan_ms += t0;
        prof->push_ms += t1;
        prof->finalize_ms += t2;
        prof->sweeps += 1;
        prof->pull_sweeps += pulling;
        pulling = p->h_bctl->pull;
        if (p->h_bctl->all_done) break;  // this sweep's finalize ended the loop, as in the graph
    }
    return DI_OK;
}

int batch_grid(const di_graph *g, long long work) {
    return (int)std::max(1LL, std::min((work + 255) / 256, (long long)g->num_sms * 8));
}

}  // namespace

// widths 4, 8, 16, 32, 64 lanes use slots 0..4
di_status pool_build_loop(di_graph *g, BatchPool *p, int slot) {
    if (p->exec[slot]) return DI_OK;
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
    const int S = p->stride ? p->stride : slot_width(slot);
    switch (slot) {
        case 0: capture_batch_body<1>(g, p, handle, S); break;
        case 1: capture_batch_body<2>(g, p, handle, S); break;
        case 2: capture_batch_body<4>(g, p, handle, S); break;
        case 3: capture_batch_body<8>(g, p, handle, S); break;
        default: capture_batch_body<16>(g, p, handle, S); break;
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(g->cap, &captured);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaStreamEndCapture"); }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphInstantiate(batch)"); }
    p->graph[slot] = graph;
    p->exec[slot] = exec;
    return DI_OK;
}

long long pool_bytes(const di_graph *g, int lanes) {
    const long long rows = (long long)g->G * g->chunk, n = g->n, L = g->nnz;
    // the graph's in-link CSR, its bins and in_dst, unless an earlier call built them
    const long long tr = (g->transposed ? 0 : 4 * (n + 1) + 4 * L + 8 * n + 4 * (n + 1)) + (g->in_dst ? 0 : 4 * L);
    return lanes * (4 * rows + 12 * n) + 4 * n + 4 * rows + (long long)sizeof(int) * kCountRows * (2 * g->W + 1) +
           (long long)(sizeof(BatchQ) * kLanes + sizeof(BatchCtl)) + 256 + tr;
}

di_status pool_alloc(di_graph *g, BatchPool *p, int lanes, cudaStream_t s) {
    if (p->Fb) return DI_OK;
    {
        di_status r = build_in_dst(g);  // the in-links of the pull direction
        if (r != DI_OK) return r;
    }
    const long long rows = (long long)g->G * g->chunk;
    p->rows = rows;
    p->cap_lanes = lanes;
    DI_CUDA(cudaMallocAsync(&p->Fb, sizeof(float) * lanes * (size_t)rows, s));
    DI_CUDA(cudaMallocAsync(&p->Hb, sizeof(double) * lanes * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&p->selb_rows, sizeof(float) * lanes * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&p->selb_node, sizeof(int) * (size_t)g->n, s));
    DI_CUDA(cudaMallocAsync(&p->spos, sizeof(int) * (size_t)rows, s));
    DI_CUDA(cudaMallocAsync(&p->fcount, sizeof(int) * kCountRows * (size_t)g->W, s));
    DI_CUDA(cudaMallocAsync(&p->pre, sizeof(int) * kCountRows * (size_t)(g->W + 1), s));
    DI_CUDA(cudaMallocAsync(&p->ticket, sizeof(unsigned), s));
    DI_CUDA(cudaMallocAsync(&p->bq, sizeof(BatchQ) * kLanes, s));
    DI_CUDA(cudaMallocAsync(&p->bctl, sizeof(BatchCtl), s));
    DI_CUDA(cudaMemsetAsync(p->ticket, 0, sizeof(unsigned), s));
    DI_CUDA(cudaMallocHost(&p->h_bq, sizeof(BatchQ) * kLanes));
    DI_CUDA(cudaMallocHost(&p->h_bctl, sizeof(BatchCtl)));
    return DI_OK;
}

void pool_free(BatchPool *p, cudaStream_t s) {
    if (!p) return;
    for (int k = 0; k < kWidths; ++k) {
        if (p->exec[k]) cudaGraphExecDestroy(p->exec[k]);
        if (p->graph[k]) cudaGraphDestroy(p->graph[k]);
    }
    void *bufs[] = {p->Fb, p->Hb, p->selb_rows, p->selb_node, p->spos, p->fcount, p->pre, p->ticket, p->bq, p->bctl};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, s);
    cudaStreamSynchronize(s);
    if (p->h_bq) cudaFreeHost(p->h_bq);
    if (p->h_bctl) cudaFreeHost(p->h_bctl);
    cudaGetLastError();
    delete p;
}

// zero fluid and histories; every lane idle
di_status pool_reset(di_graph *g, BatchPool *p, int K, double beta, cudaStream_t s) {
    k_binit<<<batch_grid(g, p->rows * K), 256, 0, s>>>(p->rows, g->n, K, p->Fb, p->Hb);
    k_bctl_init<<<1, kLanes, 0, s>>>(0, p->bq, p->bctl, 1.0, 1.0 - g->d, beta, g->n, INT_MAX);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

di_status pool_seed(di_graph *g, BatchPool *p, int K, int nitems, const int *q_dev, const int *seeds_dev,
                    const double *val_dev, cudaStream_t s) {
    if (nitems <= 0) return DI_OK;
    k_bseeds<<<std::max(1, std::min(1024, (nitems + 255) / 256)), 256, 0, s>>>(nitems, K, q_dev, seeds_dev, val_dev,
                                                                           g->new_of, p->Fb);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

di_status pool_retire(di_graph *g, BatchPool *p, int K, const LaneRetire &r, cudaStream_t s) {
    if (r.count <= 0) return DI_OK;
    k_blane_retire<<<batch_grid(g, (long long)g->n * r.count), 256, 0, s>>>(r, g->n, K, g->perm, p->Hb, p->Fb);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

di_status pool_launch_round(di_graph *g, BatchPool *p, int slot, const LaneAdmin &a, int round_cap, int lane_max,
                            double beta, cudaStream_t s) {
    const int S = p->stride ? p->stride : slot_width(slot);
    k_bround_begin<<<1, kLanes, 0, s>>>(a, g->n, 1.0 - g->d, beta, round_cap, lane_max, p->bq, p->bctl);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaGraphLaunch(p->exec[slot], s));
    k_bl1_pending<<<batch_grid(g, p->rows * slot_width(slot)), 256, 0, s>>>(p->rows, S, p->Fb, p->bq);
    k_bconfirm_pending<<<1, kLanes, 0, s>>>(g->n, beta, p->bq);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(p->h_bq, p->bq, sizeof(BatchQ) * kLanes, cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaMemcpyAsync(p->h_bctl, p->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    return DI_OK;
}

di_status run_query_batch(di_graph *g, int k, const int *seed_ptr, const int *seeds, const double *w, double tol,
                          double beta, int max_sweeps, double *H_out, bool out_dev, di_stats *st_q, di_stats *st_all,
                          di_profile *prof) {
    cudaStream_t s = g->stream;
    if (!g->bp) g->bp = new BatchPool();
    BatchPool *p = g->bp;
    di_status r = pool_alloc(g, p, kLanes, s);
    if (r != DI_OK) return r;
    // the narrowest row that holds the batch (4, 8, 16, 32 or 64 queries), or the width the
    // autotuner chose for it; beta < 0 takes that width's tuned threshold schedule
    int slot = lane_slot(k);
    if (g->btune[slot].exec_slot >= 0) slot = g->btune[slot].exec_slot;
    const int K = slot_width(slot);
    if (beta < 0.0) beta = g->btune[slot].beta;
    r = pool_build_loop(g, p, slot);
    if (r != DI_OK) return r;
    const int n = g->n;
    const double omd = 1.0 - g->d;
    const long long rows = p->rows;
    // seed items (query, seed, (1-d) w / sum w) prepared on the host
    const int nitems = seed_ptr[k];
    std::vector<int> q_of(nitems);
    std::vector<double> val(nitems);
    for (int q = 0; q < k; ++q) {
        double sum = 0.0;
        for (int t = seed_ptr[q]; t < seed_ptr[q + 1]; ++t) sum += w ? w[t] : 1.0;
        for (int t = seed_ptr[q]; t < seed_ptr[q + 1]; ++t) {
            q_of[t] = q;
            val[t] = omd * (w ? w[t] : 1.0) / sum;
        }
    }
    int *d_q = nullptr, *d_seeds = nullptr;
    double *d_val = nullptr;
    DI_CUDA(cudaMallocAsync(&d_q, sizeof(int) * nitems, s));
    DI_CUDA(cudaMallocAsync(&d_seeds, sizeof(int) * nitems, s));
    DI_CUDA(cudaMallocAsync(&d_val, sizeof(double) * nitems, s));
    DI_CUDA(cudaMemcpyAsync(d_q, q_of.data(), sizeof(int) * nitems, cudaMemcpyHostToDevice, s));
    DI_CUDA(cudaMemcpyAsync(d_seeds, seeds, sizeof(int) * nitems, cudaMemcpyHostToDevice, s));
    DI_CUDA(cudaMemcpyAsync(d_val, val.data(), sizeof(double) * nitems, cudaMemcpyHostToDevice, s));
    DI_CUDA(cudaEventRecord(g->ev0, s));
    const int grid = batch_grid(g, rows * K);
    k_binit<<<grid, 256, 0, s>>>(rows, n, K, p->Fb, p->Hb);
    k_bseeds<<<std::max(1, std::min(1024, (nitems + 255) / 256)), 256, 0, s>>>(nitems, K, d_q, d_seeds, d_val,
                                                                           g->new_of, p->Fb);
    k_bctl_init<<<1, kLanes, 0, s>>>(k, p->bq, p->bctl, tol, omd, beta, n, max_sweeps);
    DI_CUDA(cudaGetLastError());
    int attempts = 0;
    if (prof) {
        *prof = di_profile{};
        DI_CUDA(cudaMemcpyAsync(p->h_bctl, p->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
    }
    for (int attempt = 0; attempt < 8; ++attempt) {
        ++attempts;
        if (prof) {
            di_status pr = profile_batch_loop(g, p, slot, K, s, prof);
            if (pr != DI_OK) return pr;
        } else {
            DI_CUDA(cudaGraphLaunch(p->exec[slot], s));
        }
        k_bzero_exact<<<1, kLanes, 0, s>>>(p->bq);
        k_bl1_exact<<<grid, 256, 0, s>>>(rows, K, K, p->Fb, p->bq);
        k_bconfirm<<<1, kLanes, 0, s>>>(n, p->bq, p->bctl);
        DI_CUDA(cudaGetLastError());
        DI_CUDA(cudaMemcpyAsync(p->h_bctl, p->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        if (p->h_bctl->all_done != 0) break;
    }
    DI_CUDA(cudaEventRecord(g->ev1, s));
    if (H_out) {
        double *dst = H_out, *tmp = nullptr;
        if (!out_dev) {
            DI_CUDA(cudaMallocAsync(&tmp, sizeof(double) * (size_t)n * k, s));
            dst = tmp;
        }
        k_bgather<<<std::max(1, std::min((n + kGatherTile - 1) / kGatherTile, g->num_sms * 8)), 256, 0, s>>>(
            n, k, K, g->new_of, p->Hb, dst);
        DI_CUDA(cudaGetLastError());
        if (tmp) {
            DI_CUDA(cudaMemcpyAsync(H_out, tmp, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(tmp, s);
        }
    }
    DI_CUDA(cudaMemcpyAsync(p->h_bq, p->bq, sizeof(BatchQ) * kLanes, cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(d_q, s);
    cudaFreeAsync(d_seeds, s);
    cudaFreeAsync(d_val, s);
    float ms = 0.f;
    DI_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    const BatchCtl &c = *p->h_bctl;
    bool all_conv = true;
    for (int q = 0; q < k; ++q) {
        const BatchQ &b = p->h_bq[q];
        const bool conv = b.done == 1 && b.l1_exact <= b.tolR;
        all_conv &= conv;
        if (st_q) {
            st_q[q].bound = b.l1_exact / omd;
            st_q[q].l1_F = b.l1_exact;
            st_q[q].R = b.R;
            st_q[q].edges_pushed = c.edges;
            st_q[q].sources_pushed = c.srcs;
            st_q[q].sweeps = c.sweeps;
            st_q[q].converged = conv ? 1 : 0;
            st_q[q].seconds = ms * 1e-3;
            st_q[q].kernel_launches = 0;
        }
    }
    if (st_all) {
        double worst = 0.0;
        for (int q = 0; q < k; ++q) worst = std::max(worst, p->h_bq[q].l1_exact / omd);
        st_all->bound = worst;
        st_all->l1_F = worst * omd;
        st_all->R = 0.0;
        st_all->edges_pushed = c.edges;
        st_all->sources_pushed = c.srcs;
        st_all->sweeps = c.sweeps;
        st_all->converged = all_conv ? 1 : 0;
        st_all->seconds = ms * 1e-3;
        // init (3), scan + push + pull + finalize per loop body, confirmation (3) per attempt, gather
        st_all->kernel_launches = 3 + 4LL * c.body_runs + 3LL * attempts + (H_out ? 1 : 0);
    }
    if (c.all_done == 2 || !all_conv) return set_error(DI_ENOTCONVERGED, "a batched query stopped at a limit");
    return DI_OK;
}

}  // namespace diter
