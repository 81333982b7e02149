// push.cu -- the push of a threshold sweep: along every out-link of the nodes the
// scan selected, F_j += d * sent / outdeg(i) (the inner loop of ALGO-REF, Section 2.2).
//
// The scan (sweep.cu) has already taken each selected node's fluid out of F and added
// it to H, and listed the nodes with children per out-degree class, in ascending id,
// at per-warp offsets; this kernel spreads those lists over the whole grid.
#include <cuda_runtime.h>

#include "dbg.cuh"
#include "device_common.cuh"
#include "internal.h"

namespace diter {
namespace {

constexpr int kPushWaitLimit = 1 << 20;  // polls of a stage's mbarrier while draining after a timeout

// One elementary step F_j += w.  Edges into the hot targets (the most-linked-to
// nodes, internal ids 0..n_hot-1) are summed in the CTA's shared memory: on
// power-law graphs a single target can receive a few percent of all pushes, and
// same-address reductions serialize in one L2 slice.
// (n: the node count, read only by the index check of the DI_DEBUG build)
template <typename FT>
__device__ __forceinline__ void push_one(FT *__restrict__ F, FT *hot, int n_hot, int n, int c, FT w,
                                         unsigned long long pol) {
    (void)n;
    if (!DI_CHECK(c >= 0 && c < n, 4, c)) return;
    if (c >= n_hot) red_add(F + c, w, pol);
    else atomicAdd(hot + c, w);
}

// Rows of the warp and CTA classes: the head up to a 16-byte boundary, then int4
// loads two at a time (all loads of a step are issued before its reductions),
// then the tail.
template <typename FT>
__device__ __forceinline__ void push_row_lanes(const int *__restrict__ col_idx, FT *__restrict__ F, FT *hot, int n_hot,
                                               int n, int beg, int deg, FT w, int lane, int width,
                                               unsigned long long pol) {
    const int head = min(deg, (4 - (beg & 3)) & 3);
    if (lane < head) push_one(F, hot, n_hot, n, __ldg(col_idx + beg + lane), w, pol);
    const int body = (deg - head) >> 2;
    const int4 *v4 = reinterpret_cast<const int4 *>(col_idx + beg + head);
    int k = lane;
    for (; k + width < body; k += 2 * width) {
        const int4 q = __ldg(v4 + k);
        const int4 r = __ldg(v4 + k + width);
        push_one(F, hot, n_hot, n, q.x, w, pol);
        push_one(F, hot, n_hot, n, q.y, w, pol);
        push_one(F, hot, n_hot, n, q.z, w, pol);
        push_one(F, hot, n_hot, n, q.w, w, pol);
        push_one(F, hot, n_hot, n, r.x, w, pol);
        push_one(F, hot, n_hot, n, r.y, w, pol);
        push_one(F, hot, n_hot, n, r.z, w, pol);
        push_one(F, hot, n_hot, n, r.w, w, pol);
    }
    if (k < body) {
        const int4 q = __ldg(v4 + k);
        push_one(F, hot, n_hot, n, q.x, w, pol);
        push_one(F, hot, n_hot, n, q.y, w, pol);
        push_one(F, hot, n_hot, n, q.z, w, pol);
        push_one(F, hot, n_hot, n, q.w, w, pol);
    }
    const int t = head + 4 * body + lane;
    if (t < deg) push_one(F, hot, n_hot, n, __ldg(col_idx + beg + t), w, pol);
}

// The list offsets of one row of a sweep's lists, in the two levels the scan writes into pre:
//   pre[(L-1) G + b]   the total of row L over scan CTA b (L = 1 .. kCountRows-1),
//   pre[L W + 8b + k]  the offset of sub-chunk 8b + k (warp k of CTA b) within CTA b's part.
// Each push CTA turns the CTA totals into an exclusive prefix per row in shared memory
// (cta[b], the row's total at cta[G]); sub-chunk g's offset is cta[g / 8] plus its local one.
struct ListOffs {
    const int *cta;  // shared: G + 1 entries
    const int *loc;  // global: W = 8G entries
    int W;
    __device__ int total() const { return cta[W >> 3]; }
    __device__ int at(int g) const { return g < W ? cta[g >> 3] + __ldg(loc + g) : total(); }
    // the sub-chunk holding item t < total: the last g with at(g) <= t (the CTA by a binary
    // search in shared memory, then the warp among the CTA's eight offsets)
    __device__ int find(int t) const {
        int lo = 0, hi = W >> 3;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cta[mid] <= t) lo = mid; else hi = mid;
        }
        const int r = t - cta[lo];
        const int4 *p = reinterpret_cast<const int4 *>(loc + 8 * lo);
        const int4 x = __ldg(p), y = __ldg(p + 1);
        const int k = (x.y <= r) + (x.z <= r) + (x.w <= r) + (y.x <= r) + (y.y <= r) + (y.z <= r) + (y.w <= r);
        return 8 * lo + k;
    }
    // the same, knowing the answer is at least lo: a few steps forward, then a search
    __device__ int find_from(int t, int lo) const {
        for (int k = 0; k < 4; ++k) {
            if (at(lo + 1) > t) return lo;
            ++lo;
        }
        return find(t);
    }
};

// Walks the hub chunks [c0, c1) of a sweep in order (every thread of a CTA holds the same
// state).  Chunks are numbered sub-chunk by sub-chunk through the prefix sums of the scan's per
// warp chunk counts (pch), then entry by entry within a sub-chunk's list-3 region; an entry's
// chunk count is in its Sel record.  A chunk is a stretch of one hub row: start, length and
// the weight d*sent/outdeg of that row.
template <typename FT>
struct HubWalk {
    const RowRec<FT> *rec;
    const Sel<FT> *sel;
    const int *r3, *f3;
    ListOffs pch;
    int g, e, e_end, cum, nc, beg, deg, clen;
    FT w;
    __device__ void load_entry() {
        const Sel<FT> x = sel[e];
        const RowRec<FT> rr = rec[x.node];
        nc = x.pad;
        beg = rr.beg;
        deg = rr.deg;
        clen = hub_chunk_len(deg, nc);
        w = x.sent * rr.inv;
    }
    // position on chunk c (the first chunk this CTA takes)
    __device__ void start(int c) {
        g = pch.find(c);
        e = __ldg(r3 + g);
        e_end = e + __ldcg(f3 + g);
        cum = pch.at(g);
        load_entry();
        while (cum + nc <= c) {  // the sub-chunk's entries hold chunk c
            cum += nc;
            ++e;
            load_entry();
        }
    }
    // the next chunk after c - 1: the same entry, the next entry, or the first of a later sub-chunk
    __device__ void advance_to(int c) {
        while (c >= cum + nc) {
            cum += nc;
            if (++e >= e_end) {
                do {
                    ++g;
                } while (__ldcg(f3 + g) == 0);
                e = __ldg(r3 + g);
                e_end = e + __ldcg(f3 + g);
            }
            load_entry();
        }
    }
    __device__ void chunk(int c, int &cb, int &cl, FT &cw) const {
        const int off = (c - cum) * clen;
        cb = beg + off;
        cl = min(clen, deg - off);
        cw = w;
    }
};

// The push.  The selected nodes with children of each class are numbered 0..total-1
// through the prefix sums of the scan.  The middle class (a warp per node) is strided
// over the warps, which spreads heavy rows evenly whatever the id order (R-MAT puts its
// heaviest rows on the lowest ids), and the smallest class (a lane per node, four in
// flight, at most 8 out-links each) is split into even rank ranges per warp.  The largest
// class comes first: its rows (up to 50,000 out-links on the Zipf workload) are cut into
// chunks of kHubChunk out-links spread over the CTAs and their warps, so no CTA carries a
// whole hub.  The scan already moved each node's fluid into H; the push adds d*sent/outdeg(i)
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
    __shared__ __align__(128) int s_hcol[kWarps][kHubChunk + 8];  // a hub chunk's column indices, per warp
    __shared__ __align__(8) unsigned long long s_hbar[kWarps];
    extern __shared__ int s_cta[];  // kCountRows-1 rows of G+1: the CTA-level list offsets
    if (st->done || st->pull) return;
#ifdef DI_DEBUG
    const int n = st->n;
#else
    const int n = 0;
#endif
    constexpr int R = kCountRows - 1;
    for (int t = threadIdx.x; t < kHotSlots; t += kScanThreads) hot[t] = (FT)0;
    for (int i = threadIdx.x; i < R * G; i += kScanThreads) {
        const int r = i / G;
        s_cta[r * (G + 1) + (i - r * G)] = __ldg(pre + i);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < R) {  // warp w: exclusive prefix of row w + 1's CTA totals, in place; the total at [G]
        int *t = s_cta + w * (G + 1);
        const int per = (G + 31) / 32, b0 = min(G, lane * per), b1 = min(G, b0 + per);
        int a = 0;
        for (int b = b0; b < b1; ++b) a += t[b];
        int x = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) t[G] = x;
        int run = x - a;
        for (int b = b0; b < b1; ++b) {
            const int c = t[b];
            t[b] = run;
            run += c;
        }
    }
    __syncthreads();
    auto offs = [&](int L) { return ListOffs{s_cta + (L - 1) * (G + 1), pre + L * W, W}; };
    const unsigned long long pol = evict_last_policy(), pol_col = evict_first_policy();
    const int wait_polls = st->wait_polls;
    const int nwarps = gridDim.x * kWarps, gw = blockIdx.x * kWarps + w;
    long long edges = 0;
    // class 3: the hub rows, cut into chunks of at most kHubChunk out-links.  CTA b takes the
    // contiguous chunk range [b nch / grid, (b+1) nch / grid) and its warps take every 8th chunk
    // of it.  A chunk's column indices are staged in the warp's shared memory by a 1-D bulk copy
    // (TMA); the next chunk is located (its list entry and row record) while the copy is in
    // flight.  A CTA per hub row, or the whole CTA on one chunk at a time, left the chunks'
    // dependent loads on the critical path: slower on R-MAT, whose dense sweeps list thousands
    // of hub rows.  The hubs go first: their per-link weights d*sent/outdeg are the smallest,
    // and with FP32 fluid a small weight added after the larger ones of the other classes is
    // rounded away more often (R-MAT 2^23: 1.5e-7 against 6e-7 in L1 from FP64).
    {
        const ListOffs pch = offs(kChunkRow);
        const int nch = pch.total();
        const int cb0 = (int)((long long)blockIdx.x * nch / gridDim.x);
        const int cb1 = (int)((long long)(blockIdx.x + 1) * nch / gridDim.x);
        int c = cb0 + w;
        if (c < cb1) {
            HubWalk<FT> hw{rec, sel, region + 3 * (W + 1), fcount + 3 * W, pch};
            hw.start(c);
            const unsigned bar = smem_addr(&s_hbar[w]);
            int *stage = s_hcol[w];
            // a copy covers [beg & ~3, (beg + len + 3) & ~3): 16-byte aligned at both ends, inside
            // the column array (kColPad ints are allocated past its end); a chunk longer than the
            // stage (a row of more than kMaxHubChunks * kHubChunk links) is read directly instead
            auto issue = [&](int beg, int len) {
                if (len > kHubChunk) {
                    mbar_expect_tx(bar, 0u);
                    return;
                }
                const int a0 = beg & ~3, a1 = (beg + len + 3) & ~3;
                mbar_expect_tx(bar, 4u * (unsigned)(a1 - a0));
                bulk_copy(smem_addr(stage), col_idx + a0, 4u * (unsigned)(a1 - a0), bar, pol_col);
            };
            if (lane == 0) {
                mbar_init(bar, 1);
                fence_barrier_init();
            }
            __syncwarp();
            int cb, cl;
            FT cw;
            hw.chunk(c, cb, cl, cw);
            if (lane == 0) issue(cb, cl);
            bool ok = true;
            unsigned phase = 0;
            while (c < cb1) {
                const int nx = c + kWarps;
                int nb = 0, nl = 0;
                FT nw = (FT)0;
                if (nx < cb1) {  // the next chunk's entry and record, while this copy lands
                    hw.advance_to(nx);
                    hw.chunk(nx, nb, nl, nw);
                }
                ok = __all_sync(kFull, mbar_wait(bar, phase, wait_polls));
                if (!ok) break;
                phase ^= 1u;
                if (lane == 0) edges += cl;
                if (cl > kHubChunk) {
                    push_row_lanes(col_idx, F, hot, n_hot, n, cb, cl, cw, lane, 32, pol);
                } else {
                    const int *cols = stage + (cb & 3);
                    for (int j = lane; j < cl; j += 32) push_one(F, hot, n_hot, n, cols[j], cw, pol);
                }
                __syncwarp();  // every lane is done with the stage
                c = nx;
                if (c < cb1) {
                    cb = nb;
                    cl = nl;
                    cw = nw;
                    if (lane == 0) {
                        fence_proxy_async();
                        issue(cb, cl);
                    }
                }
            }
            if (!ok && lane == 0) {
                // the copy did not land in time: wait (bounded again) for it, then stop the solve
                // (DI_ETIMEOUT), or mark the graph untrusted if it never lands
                const bool drained = mbar_wait(bar, phase, kPushWaitLimit);
                atomicOr(reinterpret_cast<unsigned long long *>(&part[blockIdx.x % G].err), drained ? 1ull : 3ull);
            }
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
        const ListOffs p2 = offs(2);
        const int *r2 = region + 2 * (W + 1);
        const int tot = p2.total();
        for (long long k0 = 0; gw + k0 * nwarps < tot; k0 += 32) {
            const long long t = gw + (k0 + lane) * nwarps;
            int mb = 0, md = 0;
            FT mw = (FT)0;
            if (t < tot) {
                const int mg = p2.find((int)t);
                const int pos = __ldg(r2 + mg) + ((int)t - p2.at(mg));
                if (DI_CHECK(pos < __ldg(r2 + mg + 1), 2, pos)) {
                    const Sel<FT> e = sel[pos];
                    if (DI_CHECK(e.node >= 0 && e.node < n, 3, e.node)) {
                        const RowRec<FT> rr = rec[e.node];
                        mb = rr.beg;
                        md = rr.deg;
                        mw = e.sent * rr.inv;
                        edges += md;
                    }
                }
            }
            const int m = (int)min(32LL, (tot - gw - k0 * nwarps + nwarps - 1) / nwarps);
            // two nodes at a time, one per half-warp: a node's column loads and reductions are
            // a dependent round trip, and two halves keep two of them in flight
            const int half = lane >> 4;
            for (int j = 0; j < m; j += 2) {
                const int src = (j + half) & 31;
                const int rb = __shfl_sync(kFull, mb, src), rd = __shfl_sync(kFull, md, src);
                const FT rw = __shfl_sync(kFull, mw, src);
                push_row_lanes(col_idx, F, hot, n_hot, n, rb, j + half < m ? rd : 0, rw, lane & 15, 16, pol);
            }
        }
    }
    {
        // class 1: a lane per node, kInFlight nodes per lane at a time (at most 8 out-links each)
        constexpr int kInFlight = 4;
        static_assert(kOutCut1 <= 8 && kInFlight == 4, "class-1 rows are pushed in two groups of four links");
        const ListOffs p1 = offs(1);
        const int *r1 = region + 1 * (W + 1);
        const int tot = p1.total();
        const int per = (tot + nwarps - 1) / nwarps;
        const int t_beg = min(tot, gw * per), t_end = min(tot, t_beg + per);
        int gs = 0;
        if (t_beg < t_end) {
            if (lane == 0) gs = p1.find(t_beg);
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
                    mg = p1.find_from(t, mg);
                    pos[u] = __ldg(r1 + mg) + (t - p1.at(mg));
                    if (!DI_CHECK(pos[u] < __ldg(r1 + mg + 1), 2, pos[u])) pos[u] = -1;
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
                    if (!DI_CHECK(e.node >= 0 && e.node < n, 3, e.node)) pos[u] = -1;
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
                    if (k < rd[u]) push_one(F, hot, n_hot, n, cc[u][k], rw[u], pol);
            if (__any_sync(kFull, rd[0] > 4 || rd[1] > 4 || rd[2] > 4 || rd[3] > 4)) {
#pragma unroll
                for (int u = 0; u < kInFlight; ++u)
#pragma unroll
                    for (int k = 0; k < 4; ++k) cc[u][k] = k + 4 < rd[u] ? __ldg(col_idx + rb[u] + 4 + k) : 0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int u = 0; u < kInFlight; ++u)
                        if (k + 4 < rd[u]) push_one(F, hot, n_hot, n, cc[u][k], rw[u], pol);
            }
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
#ifdef DI_DEBUG
    const int n = st->n;
    // a link whose endpoints are outside [0, n) is dropped (src = dst = -1, as past the range)
    auto check_link = [&](int &s, int &d, long long e) {
        if (s >= 0 && !DI_CHECK(s < n && d >= 0 && d < n, 5, e)) s = d = -1;
    };
#endif
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
#ifdef DI_DEBUG
                check_link(src[u], dst[u], e);
#endif
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
#ifdef DI_DEBUG
#pragma unroll
            for (int k = 0; k < kPullRun; ++k) check_link(src[k], dst[k], eb + k);
#endif
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

// the push's dynamic shared memory: the CTA-level list offsets of kCountRows-1 rows
inline size_t push_dyn_smem(const di_graph *g) { return sizeof(int) * (kCountRows - 1) * (size_t)(g->G + 1); }

// allows the largest dynamic shared memory the push can take (G <= kMaxScanBlocks) on the
// current device; called before a sweep loop is captured
di_status push_setup() {
    const int bytes = (int)(sizeof(int) * (kCountRows - 1) * (size_t)(kMaxScanBlocks + 1));
    DI_CUDA(cudaFuncSetAttribute(k_sweep_push<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    DI_CUDA(cudaFuncSetAttribute(k_sweep_push<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return DI_OK;
}

template <typename FT>
void launch_push(di_graph *g, FT *F, cudaStream_t s) {
    k_sweep_push<FT><<<push_grid(g), kScanThreads, push_dyn_smem(g), s>>>(rec_of<FT>(g), g->col_idx, F, g->region, g->pre,
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

#ifdef DI_DEBUG
unsigned long long dbg_take_push() { return dbg_take_word(); }
#endif

template void launch_pull<double>(di_graph *, double *, cudaStream_t);
template void launch_pull<float>(di_graph *, float *, cudaStream_t);

}  // namespace diter
