// push.cu -- the push of a threshold sweep: along every out-link of the nodes the
// scan selected, F_j += d * sent / outdeg(i) (the inner loop of ALGO-REF, Section 2.2).
//
// The scan (sweep.cu) has already taken each selected node's fluid out of F and added
// it to H, and listed the nodes with children per out-degree class, in ascending id,
// at per-warp offsets; this kernel spreads those lists over the whole grid.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace diter {
namespace {

constexpr int kPushWaitLimit = 1 << 20;  // polls of a stage's mbarrier while draining after a timeout

// One elementary step F_j += w.  Edges into the hot targets (the most-linked-to
// nodes, internal ids 0..n_hot-1) are summed in the CTA's shared memory: on
// power-law graphs a single target can receive a few percent of all pushes, and
// same-address reductions serialize in one L2 slice.
template <typename FT>
__device__ __forceinline__ void push_one(FT *__restrict__ F, FT *hot, int n_hot, int c, FT w,
                                         unsigned long long pol) {
    if (c >= n_hot) red_add(F + c, w, pol);
    else atomicAdd(hot + c, w);
}

// Rows of the warp and CTA classes: the head up to a 16-byte boundary, then int4
// loads two at a time (all loads of a step are issued before its reductions),
// then the tail.
template <typename FT>
__device__ __forceinline__ void push_row_lanes(const int *__restrict__ col_idx, FT *__restrict__ F, FT *hot, int n_hot,
                                               int beg, int deg, FT w, int lane, int width, unsigned long long pol) {
    const int head = min(deg, (4 - (beg & 3)) & 3);
    if (lane < head) push_one(F, hot, n_hot, __ldg(col_idx + beg + lane), w, pol);
    const int body = (deg - head) >> 2;
    const int4 *v4 = reinterpret_cast<const int4 *>(col_idx + beg + head);
    int k = lane;
    for (; k + width < body; k += 2 * width) {
        const int4 q = __ldg(v4 + k);
        const int4 r = __ldg(v4 + k + width);
        push_one(F, hot, n_hot, q.x, w, pol);
        push_one(F, hot, n_hot, q.y, w, pol);
        push_one(F, hot, n_hot, q.z, w, pol);
        push_one(F, hot, n_hot, q.w, w, pol);
        push_one(F, hot, n_hot, r.x, w, pol);
        push_one(F, hot, n_hot, r.y, w, pol);
        push_one(F, hot, n_hot, r.z, w, pol);
        push_one(F, hot, n_hot, r.w, w, pol);
    }
    if (k < body) {
        const int4 q = __ldg(v4 + k);
        push_one(F, hot, n_hot, q.x, w, pol);
        push_one(F, hot, n_hot, q.y, w, pol);
        push_one(F, hot, n_hot, q.z, w, pol);
        push_one(F, hot, n_hot, q.w, w, pol);
    }
    const int t = head + 4 * body + lane;
    if (t < deg) push_one(F, hot, n_hot, __ldg(col_idx + beg + t), w, pol);
}

// Enumerate the class-3 (hub) entries of the sweep and cut their rows into chunks of
// kHubChunk out-links: every CTA builds the same table in shared memory -- the list
// position of each entry (s_pos) and the exclusive prefix sums of the chunk counts
// (s_pre, te + 1 values) -- from the per-warp list counts of the scan.  Thread t takes the
// sub-chunks t, t + 256, ...; entries are numbered thread by thread, so the enumeration
// is the same in every CTA.  te is the class's list total (the caller checks te <= kHubCap);
// it receives the number of entries in the table.  Returns the number of chunks (valid in
// every thread).
template <typename FT>
__device__ int hub_chunks(const RowRec<FT> *__restrict__ rec, const Sel<FT> *__restrict__ sel,
                          const int *__restrict__ region, const int *__restrict__ fcount, int W, int &te,
                          int *s_pos, int *s_pre, int *s_scan) {
    const int *r3 = region + 3 * (W + 1), *f3 = fcount + 3 * W;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // 1. entries per thread, an exclusive block scan, then each thread lists its entries
    int ents = 0;
#pragma unroll 4
    for (int gg = threadIdx.x; gg < W; gg += kScanThreads) ents += __ldcg(f3 + gg);
    int x = ents;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[w] = x;
    __syncthreads();
    int oe = x - ents, listed = 0;
    for (int k = 0; k < kWarps; ++k) {
        oe += k < w ? s_scan[k] : 0;
        listed += s_scan[k];
    }
    te = min(te, listed);  // the same count as the list total; never more than the table holds
    if (ents) {
        for (int gg = threadIdx.x; gg < W; gg += kScanThreads) {
            const int c = __ldcg(f3 + gg);
            const int b = c ? __ldg(r3 + gg) : 0;
            for (int k = 0; k < c; ++k, ++oe)
                if (oe < te) s_pos[oe] = b + k;
        }
    }
    __syncthreads();
    // 2. chunks of every entry
    for (int e = threadIdx.x; e < te; e += kScanThreads) {
        const int deg = rec[sel[s_pos[e]].node].deg;
        s_pre[e] = (deg + kHubChunk - 1) / kHubChunk;
    }
    __syncthreads();
    // 3. exclusive prefix over the chunk counts: a contiguous run per thread, then a block scan
    const int per = (te + kScanThreads - 1) / kScanThreads;
    const int e0 = min(te, (int)threadIdx.x * per), e1 = min(te, e0 + per);
    int run = 0;
    for (int e = e0; e < e1; ++e) run += s_pre[e];
    x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();  // every thread has read s_scan of step 1
    if (lane == 31) s_scan[w] = x;
    __syncthreads();
    int off = x - run, total = 0;
    for (int k = 0; k < kWarps; ++k) {
        off += k < w ? s_scan[k] : 0;
        total += s_scan[k];
    }
    for (int e = e0; e < e1; ++e) {
        const int c = s_pre[e];
        s_pre[e] = off;
        off += c;
    }
    if (threadIdx.x == 0) s_pre[te] = total;
    __syncthreads();
    return total;
}

// The push.  The selected nodes with children of each class are numbered 0..total-1
// through the prefix sums of the scan.  The middle class (a warp per node) is strided
// over the warps, which spreads heavy rows evenly whatever the id order (R-MAT puts its
// heaviest rows on the lowest ids), and the smallest class (a lane per node, four in
// flight, at most 8 out-links each) is split into even rank ranges per warp.  The largest
// class comes last: its rows (up to 50,000 out-links on the Zipf workload) are cut into
// chunks of kHubChunk out-links that are strided over the CTAs, so no CTA carries a whole
// hub.  The scan already moved each node's fluid into H; the push adds d*sent/outdeg(i)
// to F_j along every out-link (ALGO-REF's inner loop), every load of a node issued before
// its reductions.
template <typename FT>
__global__ void __launch_bounds__(kScanThreads, 4) k_sweep_push(const RowRec<FT> *__restrict__ rec,
                                                             const int *__restrict__ col_idx, FT *__restrict__ F,
                                                             const int *__restrict__ region,
                                                             const int *__restrict__ pre,
                                                             const int *__restrict__ fcount, int W,
                                                             const Sel<FT> *__restrict__ sel, int n_hot,
                                                             ScanPartial *__restrict__ part, int G,
                                                             const SolveState *__restrict__ st) {
    __shared__ FT hot[kHotSlots];
    __shared__ long long s_red[kWarps];
    __shared__ int s_idx;
    __shared__ int s_hpos[kHubCap], s_hpre[kHubCap + 1], s_scan[kWarps];
    __shared__ __align__(128) int s_hcol[2][kHubChunk + 8];  // two stages of a hub chunk's column indices
    __shared__ __align__(8) unsigned long long s_hbar[2];
    if (st->done || st->pull) return;
    for (int t = threadIdx.x; t < kHotSlots; t += kScanThreads) hot[t] = (FT)0;
    __syncthreads();
    const unsigned long long pol = evict_last_policy(), pol_col = evict_first_policy();
    const int wait_polls = st->wait_polls;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nwarps = gridDim.x * kWarps, gw = blockIdx.x * kWarps + w;
    const int *pre3 = pre + 3 * (W + 1);
    long long edges = 0;
    const int tot3 = __ldg(pre3 + W);
    if (tot3 > kHubCap) {
        // more hubs than the chunk table holds (dense sweeps of hub-rich graphs): the whole
        // CTA per node, nodes strided over the CTAs
        for (int t = blockIdx.x; t < tot3; t += gridDim.x) {
            if (threadIdx.x == 0) {
                const int gs = find_sub(pre3, W, t);
                s_idx = region[3 * (W + 1) + gs] + (t - __ldg(pre3 + gs));
            }
            __syncthreads();
            const Sel<FT> e = sel[s_idx];
            __syncthreads();
            const RowRec<FT> rr = rec[e.node];
            if (threadIdx.x == 0) edges += rr.deg;
            push_row_lanes(col_idx, F, hot, n_hot, rr.beg, rr.deg, e.sent * rr.inv, threadIdx.x, kScanThreads, pol);
        }
    }
    // classes 2 and 1: each warp takes an even range of ranks of the class's list (ranks
    // number the list entries over all sub-chunks, so the split is even however the selected
    // nodes fall over the sub-chunks); a lane finds the sub-chunk of its rank from the
    // warp's current one
    {
        // class 2: a half-warp per node, strided over the ranks (rank t to warp t mod nwarps),
        // which interleaves heavy and light rows on any id order; lane j first finds and fetches
        // the entry and row record of the warp's j-th node of each group of 32, so only the
        // column loads remain on each node's path
        const int *p2 = pre + 2 * (W + 1), *r2 = region + 2 * (W + 1);
        const int tot = __ldg(p2 + W);
        for (long long k0 = 0; gw + k0 * nwarps < tot; k0 += 32) {
            const long long t = gw + (k0 + lane) * nwarps;
            int mb = 0, md = 0;
            FT mw = (FT)0;
            if (t < tot) {
                const int mg = find_sub(p2, W, (int)t);
                const Sel<FT> e = sel[__ldg(r2 + mg) + ((int)t - __ldg(p2 + mg))];
                const RowRec<FT> rr = rec[e.node];
                mb = rr.beg;
                md = rr.deg;
                mw = e.sent * rr.inv;
                edges += md;
            }
            const int m = (int)min(32LL, (tot - gw - k0 * nwarps + nwarps - 1) / nwarps);
            // two nodes at a time, one per half-warp: a node's column loads and reductions are
            // a dependent round trip, and two halves keep two of them in flight
            const int half = lane >> 4;
            for (int j = 0; j < m; j += 2) {
                const int src = (j + half) & 31;
                const int rb = __shfl_sync(kFull, mb, src), rd = __shfl_sync(kFull, md, src);
                const FT rw = __shfl_sync(kFull, mw, src);
                push_row_lanes(col_idx, F, hot, n_hot, rb, j + half < m ? rd : 0, rw, lane & 15, 16, pol);
            }
        }
    }
    {
        // class 1: a lane per node, kInFlight nodes per lane at a time (at most 8 out-links each)
        constexpr int kInFlight = 4;
        static_assert(kOutCut1 <= 8 && kInFlight == 4, "class-1 rows are pushed in two groups of four links");
        const int *p1 = pre + 1 * (W + 1), *r1 = region + 1 * (W + 1);
        const int tot = __ldg(p1 + W);
        const int per = (tot + nwarps - 1) / nwarps;
        const int t_beg = min(tot, gw * per), t_end = min(tot, t_beg + per);
        int gs = 0;
        if (t_beg < t_end) {
            if (lane == 0) gs = find_sub(p1, W, t_beg);
            gs = __shfl_sync(kFull, gs, 0);
        }
        for (int t0 = t_beg; t0 < t_end; t0 += 32 * kInFlight) {
            // list positions first (the prefix sums stay in L1), then every entry load, then
            // every row record, so that each step has all of its loads in flight together
            int pos[kInFlight];
            int mg = gs;
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) {
                const int t = t0 + 32 * u + lane;
                pos[u] = -1;
                if (t < t_end) {
                    mg = find_sub_from(p1, W, t, mg);
                    pos[u] = __ldg(r1 + mg) + (t - __ldg(p1 + mg));
                }
            }
            // every lane's last rank is below the next group's first: restart from the largest
            gs = __reduce_max_sync(kFull, (unsigned)mg);
            int node[kInFlight];
            FT sent[kInFlight];
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) {
                node[u] = 0;
                sent[u] = (FT)0;
                if (pos[u] >= 0) {
                    const Sel<FT> e = sel[pos[u]];
                    node[u] = e.node;
                    sent[u] = e.sent;
                }
            }
            int rb[kInFlight], rd[kInFlight];
            FT rw[kInFlight];
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) {
                rb[u] = 0;
                rd[u] = 0;
                rw[u] = (FT)0;
                if (pos[u] >= 0) {
                    const RowRec<FT> rr = rec[node[u]];
                    rb[u] = rr.beg;
                    rd[u] = rr.deg;
                    rw[u] = sent[u] * rr.inv;
                }
            }
            // the first four out-links of every node (most rows have one to three), then the rest
            int cc[kInFlight][4];
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) {
                edges += rd[u];
#pragma unroll
                for (int k = 0; k < 4; ++k) cc[u][k] = k < rd[u] ? __ldg(col_idx + rb[u] + k) : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int u = 0; u < kInFlight; ++u)
                    if (k < rd[u]) push_one(F, hot, n_hot, cc[u][k], rw[u], pol);
            if (__any_sync(kFull, rd[0] > 4 || rd[1] > 4 || rd[2] > 4 || rd[3] > 4)) {
#pragma unroll
                for (int u = 0; u < kInFlight; ++u)
#pragma unroll
                    for (int k = 0; k < 4; ++k) cc[u][k] = k + 4 < rd[u] ? __ldg(col_idx + rb[u] + 4 + k) : 0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int u = 0; u < kInFlight; ++u)
                        if (k + 4 < rd[u]) push_one(F, hot, n_hot, cc[u][k], rw[u], pol);
            }
        }
    }
    // class 3: chunks of kHubChunk out-links of the hub rows, strided over the CTAs.  Each
    // chunk's column indices are staged in shared memory by a 1-D bulk copy (TMA) into one of
    // two stages, the next chunk's copy in flight while a chunk is pushed.  (Setting up the
    // table and the first copies before the other classes, so that the copies land while they
    // run, was slower: the table's dependent loads then delay every warp.)
    const bool hubs = tot3 > 0 && tot3 <= kHubCap;
    int ne = tot3, nch = 0, mine = 0;
    const int first = blockIdx.x, step = gridDim.x;
    // chunk i of this CTA: its row, start and length (the same in every thread)
    auto locate = [&](int i, int &beg, int &len, FT &wv) {
        const int t = first + i * step;
        int lo = 0, hi = ne;  // the entry holding chunk t: the last e with s_hpre[e] <= t
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_hpre[mid] <= t) lo = mid; else hi = mid;
        }
        const Sel<FT> e = sel[s_hpos[lo]];
        const RowRec<FT> rr = rec[e.node];
        const int off = (t - s_hpre[lo]) * kHubChunk;
        beg = rr.beg + off;
        len = min(kHubChunk, rr.deg - off);
        wv = e.sent * rr.inv;
    };
    // a copy covers [beg & ~3, (beg + len + 3) & ~3): 16-byte aligned at both ends, inside the
    // column array (kColPad ints are allocated past its end)
    auto issue = [&](int k, int beg, int len) {
        const int a0 = beg & ~3, a1 = (beg + len + 3) & ~3;
        const unsigned bar = smem_addr(&s_hbar[k]);
        mbar_expect_tx(bar, 4u * (unsigned)(a1 - a0));
        bulk_copy(smem_addr(s_hcol[k]), col_idx + a0, 4u * (unsigned)(a1 - a0), bar, pol_col);
    };
    int cb[2] = {0, 0}, cl[2] = {0, 0};
    FT cw[2] = {(FT)0, (FT)0};
    if (hubs) {
        __syncthreads();
        nch = hub_chunks(rec, sel, region, fcount, W, ne, s_hpos, s_hpre, s_scan);
        mine = first < nch ? (nch - 1 - first) / step + 1 : 0;  // chunks of this CTA
        if (threadIdx.x == 0 && mine > 0) {
            mbar_init(smem_addr(&s_hbar[0]), 1);
            mbar_init(smem_addr(&s_hbar[1]), 1);
            fence_barrier_init();
        }
        __syncthreads();
        for (int i = 0; i < 2 && i < mine; ++i) {
            locate(i, cb[i], cl[i], cw[i]);
            if (threadIdx.x == 0) issue(i, cb[i], cl[i]);
        }
    }
    if (hubs) {
        bool ok = true;
        int i = 0;
        for (; i < mine; ++i) {
            const int k = i & 1;
            ok = __all_sync(kFull, mbar_wait(smem_addr(&s_hbar[k]), (unsigned)((i >> 1) & 1), wait_polls));
            if (__syncthreads_or(!ok)) {
                ok = false;
                break;
            }
            const int *cols = s_hcol[k] + (cb[k] & 3);
            if (threadIdx.x == 0) edges += cl[k];
            for (int j = threadIdx.x; j < cl[k]; j += kScanThreads) push_one(F, hot, n_hot, cols[j], cw[k], pol);
            __syncthreads();  // every thread is done with stage k
            if (i + 2 < mine) {
                locate(i + 2, cb[k], cl[k], cw[k]);
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    issue(k, cb[k], cl[k]);
                }
            }
        }
        if (!ok && threadIdx.x == 0) {
            // a copy did not land in time: wait (bounded again) for the ones still in flight,
            // then stop the solve (DI_ETIMEOUT), or mark the graph untrusted if they never land
            bool drained = true;
            for (int j = i; j < mine && j < i + 2; ++j)
                drained &= mbar_wait(smem_addr(&s_hbar[j & 1]), (unsigned)((j >> 1) & 1), kPushWaitLimit);
            atomicOr(reinterpret_cast<unsigned long long *>(&part[blockIdx.x % G].err), drained ? 1ull : 3ull);
        }
    }
    // the CTA's sums for the hot targets go to F once
    __syncthreads();
    for (int t = threadIdx.x; t < n_hot; t += kScanThreads) {
        const FT v = hot[t];
        if (v != (FT)0) red_add(F + t, v);
    }
    const long long be = block_sum(edges, s_red);
    // the scan zeroed the G partials' edge counts; the push grid may be wider than G
    if (threadIdx.x == 0 && be)
        atomicAdd(reinterpret_cast<unsigned long long *>(&part[blockIdx.x % G].edges), (unsigned long long)be);
}

}  // namespace

// The pull direction of a dense sweep: the same diffusion of S read from the target side,
// F_j += sum over in-links (i -> j) of w_i, where the scan wrote w_i = sent_i * d/outdeg_i for
// the selected nodes and 0 for the others.  The in-links, in target order, are cut into
// even ranges per warp.  The out-links pushed are counted by the scan on these sweeps.
//  * FP32: lane l takes link e0 + l and a segmented warp sum over equal targets (a shuffle
//    tree) leaves one red.add per target and 32 links.
//  * FP64: FP64 arithmetic is scarce on this GPU (a shuffle tree made the pull slower than
//    the push), so each lane takes kPullRun consecutive links and sums them serially per
//    target, one add per link, then adds each target's sum with one red.add.
// Either way a target with many in-links gets a reduction per 32 or kPullRun links where
// the push makes one per link.
constexpr int kPullRun = 16;

template <typename FT>
__global__ void __launch_bounds__(kScanThreads, 3) k_sweep_pull(const int *__restrict__ in_src,
                                                             const int *__restrict__ in_dst,
                                                             const FT *__restrict__ w, long long nnz,
                                                             FT *__restrict__ F, const SolveState *__restrict__ st) {
    if (st->done || !st->pull) return;
    constexpr bool kTree = sizeof(FT) == 4;
    constexpr int kU = 4;  // shuffle tree: steps of 32 links loaded before they are summed
    constexpr int kStepLinks = kTree ? 32 * kU : 32 * kPullRun;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * kWarps, gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    // ranges of whole steps, so that every full run starts on a 32-byte boundary
    const long long per = (nnz + nwarps - 1) / nwarps + kStepLinks - 1;
    const long long span = per - per % kStepLinks;
    const long long e_beg = min(nnz, gw * span), e_end = min(nnz, e_beg + span);
    const unsigned long long pol = evict_last_policy();
    for (long long e0 = e_beg; e0 < e_end; e0 += kStepLinks) {
        if constexpr (kTree) {
            int dst[kU], src[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const long long e = e0 + 32 * u + lane;
                const bool in = e < e_end;
                dst[u] = in ? __ldg(in_dst + e) : -1;
                src[u] = in ? __ldg(in_src + e) : -1;
            }
            FT v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) v[u] = src[u] >= 0 ? __ldg(w + src[u]) : (FT)0;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                // inclusive sums over the runs of equal targets (targets ascend along the links)
                FT a = v[u];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const FT y = __shfl_up_sync(kFull, a, o);
                    const int dy = __shfl_up_sync(kFull, dst[u], o);
                    if (lane >= o && dy == dst[u]) a += y;
                }
                const int dn = __shfl_down_sync(kFull, dst[u], 1);
                const bool last = dst[u] >= 0 && (lane == 31 || dn != dst[u]);
                if (last && a != (FT)0) red_add(F + dst[u], a, pol);
            }
        } else {
            const long long eb = e0 + (long long)kPullRun * lane;
            int src[kPullRun], dst[kPullRun];
            if (eb + kPullRun <= e_end) {
                const int4 *ps = reinterpret_cast<const int4 *>(in_src + eb);
                const int4 *pd = reinterpret_cast<const int4 *>(in_dst + eb);
#pragma unroll
                for (int h = 0; h < kPullRun / 4; ++h) {
                    const int4 a = __ldg(ps + h), b = __ldg(pd + h);
                    src[4 * h] = a.x; src[4 * h + 1] = a.y; src[4 * h + 2] = a.z; src[4 * h + 3] = a.w;
                    dst[4 * h] = b.x; dst[4 * h + 1] = b.y; dst[4 * h + 2] = b.z; dst[4 * h + 3] = b.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kPullRun; ++k) {
                    const bool in = eb + k < e_end;
                    src[k] = in ? __ldg(in_src + eb + k) : -1;
                    dst[k] = in ? __ldg(in_dst + eb + k) : -1;
                }
            }
            FT v[kPullRun];
#pragma unroll
            for (int k = 0; k < kPullRun; ++k) v[k] = src[k] >= 0 ? __ldg(w + src[k]) : (FT)0;
            int cur = dst[0];
            FT acc = v[0];
#pragma unroll
            for (int k = 1; k < kPullRun; ++k) {
                if (dst[k] != cur) {
                    if (cur >= 0 && acc != (FT)0) red_add(F + cur, acc, pol);
                    cur = dst[k];
                    acc = (FT)0;
                }
                acc += v[k];
            }
            if (cur >= 0 && acc != (FT)0) red_add(F + cur, acc, pol);
        }
    }
}

template <typename FT>
void launch_push(di_graph *g, FT *F, cudaStream_t s) {
    k_sweep_push<FT><<<push_grid(g), kScanThreads, 0, s>>>(rec_of<FT>(g), g->col_idx, F, g->region, g->pre,
                                                           g->fcount, g->W, sel_of<FT>(g), g->n_hot, g->part, g->G,
                                                           g->st);
}

template void launch_push<double>(di_graph *, double *, cudaStream_t);
template void launch_push<float>(di_graph *, float *, cudaStream_t);

template <typename FT>
void launch_pull(di_graph *g, FT *F, cudaStream_t s) {
    // one wave at 3 CTAs per SM (16 gathers in flight per lane in FP64)
    k_sweep_pull<FT><<<g->num_sms * 3, kScanThreads, 0, s>>>(g->in_src, g->in_dst, static_cast<const FT *>(g->wpull),
                                                             g->nnz, F, g->st);
}

template void launch_pull<double>(di_graph *, double *, cudaStream_t);
template void launch_pull<float>(di_graph *, float *, cudaStream_t);

}  // namespace diter
