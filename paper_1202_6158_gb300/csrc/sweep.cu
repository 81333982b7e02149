// sweep.cu -- the D-iteration hot path: threshold sweeps on the device.
//
// One sweep (Section 4.2: every node whose fluid is above a threshold is
// chosen, and the threshold is lowered progressively) is three kernels:
//
//   k_sweep_scan<FT>   streams F and the one-byte out-degree class of every node
//                      (no dependent loads, no block barriers).  It sums |F|_1 in
//                      exact 64-bit fixed point, selects S = {i : |F_i| > T} (for
//                      FP64 an integer compare of the bit patterns), zeroes F_i for
//                      the selected nodes, adds sent to H_i (the J_i F step of
//                      Section 2.2, a red.add in node order) and appends (i, sent)
//                      of the nodes with children to the list of the node's class,
//                      in ascending id, with warp prefix sums; each warp writes at
//                      offsets fixed at create time, so there are no atomics.  It
//                      also sums the removed mass: (1-d)*sent for nodes with
//                      children, sent for dangling ones (Section 3.3).  Each CTA
//                      writes its list totals and its warps' offsets within them;
//                      the push builds the CTA-level prefix itself.
//   k_sweep_push<FT>   pushes d*sent/outdeg_i along every out-link (ALGO-REF's inner
//                      loop) with red.global.add; a CTA per node above kOutCut2
//                      out-links, a warp per node above kOutCut1, a lane per node
//                      otherwise; 128-bit column-index loads; the most-linked-to
//                      targets are summed in shared memory first.
//   k_sweep_finalize   one CTA reduces the per-CTA partials in fixed order,
//                      R = |F|_1 - removed, sets the next threshold
//                      T = beta*R/n (halved after an empty sweep), and stops the
//                      CUDA-graph while-loop when R <= tol*(1-d) or a limit hits.
//
// All of S gives up its fluid before any push (the scan kernel finishes before
// the push kernel starts), so a sweep is the diffusion of the set S on a
// snapshot of F: F' = (I - J_S + dPJ_S)F, H' = H + J_S F.  Theorem 1
// (H + F = F_0 + dPH) holds after every sweep by the induction of Section 3.1.
// Fluid pushed into a node of S during the push stays in F for a later sweep.
//
// The whole loop is one CUDA graph: a while-conditional node whose body is the
// three kernels, so a solve makes no host round trip per sweep.  After the loop
// the exact |F|_1 is recomputed in FP64 to confirm the stop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "dbg.cuh"
#include "device_common.cuh"
#include "internal.h"

namespace diter {
namespace {

di_status ensure_pull(di_graph *g);  // the pull direction's inputs, built at first use (below)

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
                             double one_minus_d, const int *__restrict__ new_of, FT *__restrict__ F) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nseeds; k += gridDim.x * blockDim.x) {
        double v = (w ? w[k] : 1.0) / wsum;
        atomicAdd(&F[new_of[seeds[k]]], (FT)(one_minus_d * v));
    }
}

__device__ void init_control(SolveState *st, double R0, double tolR, double beta, double one_minus_d, int n,
                             long long max_edges, int max_sweeps, int trace_on, double wscale, int weighted,
                             long long pull_edges, int wait_polls, int pause_pull) {
    st->wait_polls = wait_polls;
    st->pause_pull = pause_pull;
    st->pull = 0;  // the first two sweeps push
    st->dense = 0;
    st->pull_edges = pull_edges;
    st->wscale = wscale;
    st->weighted = weighted;
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
    st->undrained = 0;
    st->n = n;
    // the while-test of ALGO-REF comes first: nothing to do if R/(1-d) <= target already
    st->done = (R0 <= tolR) ? 1 : 0;
}

__global__ void k_init_control(SolveState *st, double R0, double tolR, double beta, double one_minus_d, int n,
                               long long max_edges, int max_sweeps, int trace_on, double wscale, int weighted,
                               long long pull_edges, int wait_polls, int pause_pull) {
    init_control(st, R0, tolR, beta, one_minus_d, n, max_edges, max_sweeps, trace_on, wscale, weighted, pull_edges,
                 wait_polls, pause_pull);
}

// the same with R_0 = |F_0|_1 summed (fixed order) from the per-CTA partials of k_l1_partials:
// a continued or updated state starts from whatever fluid it holds
__global__ void k_init_control_l1(SolveState *st, const ScanPartial *__restrict__ part, int G, double tolR,
                                  double beta, double one_minus_d, int n, long long max_edges, int max_sweeps,
                                  int trace_on, double wscale, int weighted, long long pull_edges, int wait_polls,
                                  int pause_pull) {
    if (threadIdx.x != 0) return;
    double R0 = 0.0;
    for (int c = 0; c < G; ++c) R0 += part[c].l1d;
    init_control(st, R0, tolR, beta, one_minus_d, n, max_edges, max_sweeps, trace_on, wscale, weighted, pull_edges,
                 wait_polls, pause_pull);
}

// a loop paused for the in-link CSR resumes where it stopped, its next sweep pulling
__global__ void k_resume_pull(SolveState *st) {
    if (st->done == 5) st->done = 0;
    st->pause_pull = 0;
}

// ------------------------------------------------------------------- scan

// Fixed-point fluid sums.  GB300 issues only a couple of FP64 instructions per
// clock per SM, so the per-element sums of a sweep are made on the integer pipe:
// each F_i >= 0 is turned into floor(F_i * 2^S) exactly by shifting its mantissa,
// and the 64-bit integers are added.  S is chosen per sweep from the previous
// residual R (every F_i and every partial sum is at most about R) so that the
// total stays below 2^62; the result is independent of summation order and is
// within n * 2^-S, i.e. about n * 2^-61 * R, of the exact sum.
__device__ __forceinline__ int fixed_scale(double R) {
    const long long b = __double_as_longlong(R);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;  // R < 2^(e+1)
    return 60 - e;                                   // 2R * 2^S < 2^62
}

__device__ __forceinline__ long long to_fixed(double x, int S) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    int pos = (e ? e : 1) - 1075 + S;               // x * 2^S = m * 2^pos
    if (pos > 9) pos = 9;                           // only if x > 2R, which F never is
    if (pos >= 0) return (long long)(m << pos);
    if (pos <= -64) return 0;
    return (long long)(m >> (-pos));
}

__device__ __forceinline__ long long to_fixed(float x, int S) { return to_fixed((double)x, S); }

template <typename FT>
struct ScanOps;

// FP64 fluid: the threshold test compares |F_i| with T through their bit patterns
// as integers (sign bit cleared), which orders non-negative doubles exactly like
// their values.  F is non-negative except after a graph update, whose injected
// fluid may be negative; either way the test is |F_i| > T.
template <>
struct ScanOps<double> {
    using Key = long long;
    __device__ static Key key(double T) { return __double_as_longlong(T); }
    __device__ static bool above(double f, Key k) { return (__double_as_longlong(f) & 0x7fffffffffffffffLL) > k; }
    // four consecutive values starting at a 32-byte boundary
    __device__ static void load4(const double *p, double v[4], unsigned long long pol) {
        const double2 a = ld_stream(reinterpret_cast<const double2 *>(p), pol);
        const double2 b = ld_stream(reinterpret_cast<const double2 *>(p) + 1, pol);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static void load4_shared(const unsigned char *p, double v[4]) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static void store4(double *p, const double v[4]) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

template <>
struct ScanOps<float> {
    using Key = float;
    __device__ static Key key(double T) { return (float)T; }
    __device__ static bool above(float f, Key k) { return fabsf(f) > k; }
    __device__ static void load4(const float *p, float v[4], unsigned long long pol) {
        const float4 a = ld_stream(reinterpret_cast<const float4 *>(p), pol);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ static void load4_shared(const unsigned char *p, float v[4]) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ static void store4(float *p, const float v[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

// The sweep scan streams F and the one-byte out-degree class of every node: each
// warp owns a sub-chunk of chunk/8 nodes and streams it through shared memory with
// bulk copies (TMA, 1-D), kStep = 256 nodes per step and kStages steps in flight, so
// the loads never stall on a dependency; lane i takes nodes 8i..8i+7 of a step (the
// step's fixed costs -- prefix sum, barrier wait, refill -- are spread over 8 nodes
// per lane).  The
// selected nodes (id, sent) of each class are appended to that class's list in
// ascending id order with a warp prefix sum; the lists' per-sub-chunk capacities are
// fixed at create time, so no atomics are needed.
// WGT: ALGO-OP / ALGO-OP2 selection (Section 4.3) as a weighted threshold: node i
// is selected when (float)|F_i| * w_i > (float)(T * wscale), the product in FP32.
//
// The ring of one warp: per stage 256 values of F, their 256 class bytes (and 256
// selection weights); every size is a multiple of 16 bytes and every source offset a
// multiple of 256 nodes, so every copy is 16-byte aligned.

// d/outdeg from a row record read as four ints
template <typename FT>
__device__ __forceinline__ FT rec_inv(int4 r);
template <>
__device__ __forceinline__ double rec_inv<double>(int4 r) { return __hiloint2double(r.w, r.z); }
template <>
__device__ __forceinline__ float rec_inv<float>(int4 r) { return __int_as_float(r.z); }

constexpr int kPer = kStep / 32;  // nodes per lane and step
static_assert(kPer % 4 == 0 && kStep <= 256, "groups of four nodes per lane; step positions fit a byte");

// The scan CTA's six sums at once (fixed point and counts, so exact in any order):
// warp trees, one barrier, then thread k < 6 adds value k of the eight warps.
__device__ __forceinline__ void block_sums6(long long v[6], long long (*sh)[kWarps]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = warp_sum(v[k]);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) sh[k][w] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        long long a = 0;
#pragma unroll
        for (int w2 = 0; w2 < kWarps; ++w2) a += sh[threadIdx.x][w2];
        sh[threadIdx.x][0] = a;  // read back by thread 0 after the next barrier
    }
}


template <typename FT, bool WGT>
struct ScanRing {
    static constexpr int kF = kStep * (int)sizeof(FT);
    static constexpr int kC = kStep;
    static constexpr int kW = WGT ? kStep * 4 : 0;
    static constexpr int kBytes = kF + kC + kW;
    static constexpr int kStages = WGT ? 2 : 3;
    static constexpr int kWarpBytes = kBytes * kStages;
};
constexpr int kScanWaitLimit = 1 << 20;  // polls of a stage's mbarrier before the scan gives up

template <typename FT, bool WGT>
__global__ void __launch_bounds__(kScanThreads) k_sweep_scan(int wchunk, FT *__restrict__ F,
                                                             const float *__restrict__ wsel,
                                                             const unsigned char *__restrict__ cls,
                                                             const int *__restrict__ region, int W,
                                                             int *__restrict__ fcount, int *__restrict__ pre,
                                                             Sel<FT> *__restrict__ sel,
                                                             ScanPartial *__restrict__ part,
                                                             const SolveState *__restrict__ st,
                                                             double *__restrict__ H,
                                                             const RowRec<FT> *__restrict__ rec, int n,
                                                             FT *__restrict__ wpull) {
    using Ops = ScanOps<FT>;
    using Ring = ScanRing<FT, WGT>;
    __shared__ __align__(128) unsigned char s_ring[kWarps * Ring::kWarpBytes];
    __shared__ __align__(8) unsigned long long s_bar[kWarps * Ring::kStages];
    __shared__ unsigned char s_q[kWarps][kStep];  // the selected nodes of a step, by position in the step
    __shared__ long long s_red[6][kWarps];
    __shared__ int s_cnt[kCountRows][kWarps];
    __shared__ int s_err;
    if (st->done) return;
    const typename Ops::Key key = Ops::key(st->T);
    const float tw = WGT ? (float)(st->T * st->wscale) : 0.f;
    const int S = fixed_scale(st->R);
    const bool exact = (st->sweeps % kExactEvery) == 0;  // the exact |F|_1 of this sweep's start
    // a pull sweep writes sent * d/outdeg of every node (0 if not selected) instead of the lists
    const bool pull = st->pull != 0;
    const int wlim = st->wait_polls;  // the copies still in flight after a timeout are awaited with the full limit
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int g = blockIdx.x * kWarps + w;
    const long long wbeg = (long long)g * wchunk;
    int run[kLists], start[kLists];
#pragma unroll
    for (int L = 0; L < kLists; ++L) start[L] = run[L] = region[L * (W + 1) + g];
    long long l1 = 0, s_out = 0, s_dng = 0;  // fixed point: |F|_1, fluid of selected nodes with / without children
    int srcs = 0, entries = 0;
    int hub_chunks = 0;    // chunks of the hub rows this lane listed
    long long pedges = 0;  // out-links of the selected nodes, counted here on pull sweeps
    const int nsteps = wchunk / kStep;
    const unsigned long long pol = evict_first_policy();
    // this warp's ring: lane 0 keeps kStages steps in flight
    unsigned char *ring = s_ring + w * Ring::kWarpBytes;
    unsigned char *q = s_q[w];
    const unsigned ring_s = smem_addr(ring), bar0 = smem_addr(&s_bar[w * Ring::kStages]);
    auto issue = [&](int t) {
        const int k = t % Ring::kStages;
        const unsigned bar = bar0 + 8u * k, dst = ring_s + (unsigned)(k * Ring::kBytes);
        const long long base = wbeg + (long long)t * kStep;
        mbar_expect_tx(bar, Ring::kBytes);
        bulk_copy(dst, F + base, Ring::kF, bar, pol);
        bulk_copy(dst + Ring::kF, cls + base, Ring::kC, bar, pol);
        if (WGT) bulk_copy(dst + Ring::kF + Ring::kC, wsel + base, Ring::kW, bar, pol);
    };
    if (threadIdx.x == 0) s_err = 0;
    __syncthreads();
    if (lane == 0) {
        for (int k = 0; k < Ring::kStages; ++k) mbar_init(bar0 + 8u * k, 1);
        fence_barrier_init();
        for (int t = 0; t < Ring::kStages && t < nsteps; ++t) issue(t);
    }
    __syncwarp();
    int s = 0;
    bool ok = true;
    for (; s < nsteps; ++s) {
        const int slot = s % Ring::kStages;
        ok = __all_sync(kFull, mbar_wait(bar0 + 8u * slot, (unsigned)((s / Ring::kStages) & 1), wlim));
        if (!ok) break;
        const unsigned char *stg = ring + slot * Ring::kBytes;
        const FT *stg_f = reinterpret_cast<const FT *>(stg);
        const long long step0 = wbeg + (long long)s * kStep;
        // 1. which of this lane's kPer nodes (kPer/4 groups of four) are selected; the exact |F|_1
        //    every kExactEvery sweeps; on pull sweeps sent * d/outdeg of each of them
        unsigned pm = 0;
#pragma unroll
        for (int h = 0; h < kPer / 4; ++h) {
            const int j0 = kPer * lane + 4 * h;  // position in the step of the group's first node
            FT cur[4];
            Ops::load4_shared(stg + (int)sizeof(FT) * j0, cur);
            float4 wcur = make_float4(0.f, 0.f, 0.f, 0.f);
            if (WGT) wcur = *reinterpret_cast<const float4 *>(stg + Ring::kF + Ring::kC + 4 * j0);
            const float wk[4] = {wcur.x, wcur.y, wcur.z, wcur.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool pick = WGT ? fabsf((float)cur[k]) * wk[k] > tw : Ops::above(cur[k], key);
                pm |= pick ? 1u << (4 * h + k) : 0u;
                if (exact) l1 += to_fixed(cur[k], S);
            }
            if (pull) {
                const long long i0 = step0 + j0;
                const int4 *rp = reinterpret_cast<const int4 *>(rec + i0);
                FT wv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool pk = (pm >> (4 * h + k) & 1u) != 0;
                    const int4 rr = pk && i0 + k < n ? __ldg(rp + k) : make_int4(0, 0, 0, 0);
                    wv[k] = pk ? cur[k] * rec_inv<FT>(rr) : (FT)0;
                    pedges += rr.y;
                }
                Ops::store4(wpull + i0, wv);
            }
        }
        // 2. the selected nodes of the step, in ascending position, into the warp's queue
        const int np = __popc(pm);
        int incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total) {
            if (pm) {
                int at = incl - np;
#pragma unroll
                for (int h = 0; h < kPer / 4; ++h) {
                    const unsigned gm = (pm >> (4 * h)) & 0xfu;
                    if (!gm) continue;
                    const int j0 = kPer * lane + 4 * h;
                    FT z[4];
                    Ops::load4_shared(stg + (int)sizeof(FT) * j0, z);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (gm >> k & 1u) {
                            q[at++] = (unsigned char)(j0 + k);
                            z[k] = (FT)0;           // J_i F leaves F ...
                        }
                    }
                    Ops::store4(F + step0 + j0, z);
                }
            }
            __syncwarp();
            // 3. a lane per selected node: history, removed mass, list position
            for (int r = 0; r < total; r += 32) {
                const int t = r + lane;
                const bool has = t < total;
                const int idx = has ? q[t] : 0;
                const FT v = stg_f[idx];
                const int cb = has ? stg[Ring::kF + idx] : 0;  // class byte: 2 + chunks for a hub row
                const int c = class_of_byte(cb);
                const long long node = step0 + idx;
                if (has) {
                    const long long fx = to_fixed(v, S);
                    red_add(H + node, (double)v, pol);     // ... into the history (H' = H + J_S F), evict-first
                    srcs += 1;
                    if (c == 0) {
                        s_dng += fx;            // a dangling node's fluid leaves the system (Section 3.3)
                    } else {
                        s_out += fx;
                        entries += 1;
                    }
                }
                // nodes with children go to their class's list, in ascending id
#pragma unroll
                for (int L = 1; L < kLists && !pull; ++L) {
                    const bool mine = has && c == L;
                    const unsigned bits = __ballot_sync(kFull, mine);
                    if (mine) {
                        Sel<FT> e;
                        e.node = (int)node;
                        e.pad = L == 3 ? cb - 2 : 0;  // a hub row's chunk count
                        e.sent = v;
                        const int p = run[L] + __popc(bits & lt);
                        if (DI_CHECK(p < region[L * (W + 1) + g + 1], 1, p)) sel[p] = e;
                        if (L == 3) hub_chunks += cb - 2;
                    }
                    run[L] += __popc(bits);
                }
            }
        }
        // the slot is read: lane 0 refills it with the step kStages ahead
        __syncwarp();
        if (lane == 0 && s + Ring::kStages < nsteps) {
            fence_proxy_async();
            issue(s + Ring::kStages);
        }
    }
    if (!ok) {
        // a wait gave up: wait (bounded again) for this warp's copies still in flight, then report
        // (bit 1); if that wait gives up too, copies may still land in this CTA's shared memory
        // after it returns, and the graph is no longer trusted (bit 2)
        if (lane == 0) {
            bool drained = true;
            for (int t = s; t < nsteps && t < s + Ring::kStages; ++t)
                drained &= mbar_wait(bar0 + 8u * (t % Ring::kStages), (unsigned)((t / Ring::kStages) & 1),
                                     kScanWaitLimit);
            atomicOr(&s_err, drained ? 1 : 3);
        }
        __syncwarp();
    }
    hub_chunks = __reduce_add_sync(kFull, hub_chunks);
    if (lane == 0) {
#pragma unroll
        for (int L = 0; L < kLists; ++L) {
            fcount[L * W + g] = run[L] - start[L];
            s_cnt[L][w] = run[L] - start[L];
        }
        fcount[kChunkRow * W + g] = hub_chunks;
        s_cnt[kChunkRow][w] = hub_chunks;
    }
    long long sums[6] = {l1, s_out, s_dng, (long long)srcs, (long long)entries, pull ? pedges : 0};
    block_sums6(sums, s_red);
    __syncthreads();
    if (threadIdx.x == 0) {
        ScanPartial p;
        p.l1 = s_red[0][0];
        p.out = s_red[1][0];
        p.dng = s_red[2][0];
        p.edges = s_red[5][0];  // push sweeps: 0 here, added by the push kernel
        p.srcs = s_red[3][0];
        p.entries = s_red[4][0];
        p.l1d = 0.0;
        p.err = s_err;
        part[blockIdx.x] = p;
    }
    // The list offsets, in two levels (list 0, the dangling nodes, stays empty: the scan
    // finishes those nodes itself).  For rows L = 1 .. kCountRows-1 this CTA writes its
    // total, pre[(L-1) G + b], and the offset of each of its warps within the CTA's part,
    // pre[L W + 8b + k]; the push kernel turns the CTA totals into a prefix of its own, so no
    // CTA of the scan waits for the others.  (The barrier in the sums above made s_cnt visible.)
    if (threadIdx.x < kCountRows - 1) {
        const int L = threadIdx.x + 1;
        int o[kWarps], a = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            o[k] = a;
            a += s_cnt[L][k];
        }
        int4 *dst = reinterpret_cast<int4 *>(pre + L * W + kWarps * blockIdx.x);
        dst[0] = make_int4(o[0], o[1], o[2], o[3]);
        dst[1] = make_int4(o[4], o[5], o[6], o[7]);
        pre[(L - 1) * (int)gridDim.x + blockIdx.x] = a;
    }
}
static_assert(kWarps == 8, "a CTA's eight warp offsets of a row are stored as two int4");

// the bounded wait of the scan on a barrier that nothing completes: every CTA must give up
__global__ void k_selftest_wait(int polls, int *__restrict__ gave_up) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);  // one arrival completes phase 0; none ever comes
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = __all_sync(kFull, mbar_wait(b, 0u, polls));
    if (threadIdx.x == 0 && !ok) atomicAdd(gave_up, 1);
}

// --------------------------------------------------------------- finalize

__global__ void k_sweep_finalize(int n, int G, const ScanPartial *__restrict__ part, SolveState *__restrict__ st,
                                 di_sweep_record *__restrict__ trace, cudaGraphConditionalHandle handle,
                                 int in_graph) {
    __shared__ long long s_l[7][kScanThreads / 32];
    // the control block, copied by the first threads while all of them read the partials, so
    // that thread 0's bookkeeping below reads shared memory; written back once at the end
    __shared__ SolveState s_st;
    constexpr int kStWords = (int)(sizeof(SolveState) / sizeof(unsigned long long));
    static_assert(sizeof(SolveState) % sizeof(unsigned long long) == 0, "copied in 8-byte words");
    if ((int)threadIdx.x < kStWords)
        reinterpret_cast<unsigned long long *>(&s_st)[threadIdx.x] =
            reinterpret_cast<const unsigned long long *>(st)[threadIdx.x];
    // the six sums of the per-CTA partials and the OR of their error bits, reduced together:
    // warp trees, then thread 0 over the warps (integers, so exact in any order)
    long long v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
        const ScanPartial p = part[c];
        v[0] += p.l1;
        v[1] += p.out;
        v[2] += p.dng;
        v[3] += p.edges;
        v[4] += p.srcs;
        v[5] += p.entries;
        v[6] |= p.err;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += __shfl_down_sync(kFull, v[k], o);
        v[6] |= __shfl_down_sync(kFull, v[6], o);  // the error bits are OR-ed, not added
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 7; ++k) s_l[k][wid] = v[k];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    SolveState &L = s_st;
    if (L.done) {  // converged before this body ran: leave the loop
        st->body_runs = L.body_runs + 1;
        if (in_graph) cudaGraphSetConditional(handle, 0);
        return;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        long long a = 0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a = k < 6 ? a + s_l[k][w2] : (a | s_l[k][w2]);
        v[k] = a;
    }
    const long long fl1 = v[0], fout = v[1], fdng = v[2], ed = v[3], sr = v[4], en = v[5], er = v[6];
    L.body_runs += 1;
    const double Tused = L.T;
    const int S = fixed_scale(L.R);  // the scale the scan used (L.R is still the previous residual)
    // every kExactEvery sweeps the scan summed all of F; in between |F|_1 is the previous
    // residual (the removed masses are exact, only the pushes' roundings separate them)
    const bool exact = (L.sweeps % kExactEvery) == 0;
    const double l1 = exact ? ldexp((double)fl1, -S) : L.R;
    // removed mass: (1-d)*sent for nodes with children, sent for dangling nodes (Section 3.3)
    const double rem = L.one_minus_d * ldexp((double)fout, -S) + ldexp((double)fdng, -S);
    const double R = l1 - rem;  // |F|_1 after the sweep (exact arithmetic)
    const int pulled = L.pull;
    L.sweeps += 1;
    L.edges += ed;
    L.srcs += sr;
    // the next sweep pulls after two dense sweeps in a row: one dense sweep (the first sweep from
    // a uniform F_0 selects every node) is often followed by sparse ones
    const int dense = ed >= L.pull_edges ? 1 : 0;
    L.pull = dense && L.dense ? 1 : 0;
    L.dense = dense;
    if (L.trace_on && L.sweeps <= kTraceCap) {
        di_sweep_record r;
        r.l1_F = l1;
        r.removed = rem;
        r.R = R;
        r.T = Tused;
        r.sources = sr;
        r.edges = ed;
        r.pushed = en;
        r.scan_ms = 0.0;
        r.push_ms = 0.0;
        r.pull = pulled;
        r.pad = 0;
        trace[L.sweeps - 1] = r;
    }
    L.R = R;
    // T = beta R/n, halved after an empty sweep; with weights (ALGO-OP) it is never raised
    double Tn = (sr == 0) ? 0.5 * Tused : L.beta * R / (double)n;
    if (sr != 0 && L.weighted) Tn = fmin(Tused, Tn);
    if (!(Tn > 0.0)) Tn = 0.0;
    L.T = Tn;
    int done = 0;
    if (er) {
        done = 4;
        if (er & 2) L.undrained = 1;
    } else if (!isfinite(R)) done = 3;
    else if (R <= L.tolR) done = 1;
    else if (L.sweeps >= L.max_sweeps || (L.max_edges > 0 && L.edges >= L.max_edges)) done = 2;
    else if (L.pull && L.pause_pull) done = 5;  // a pull is due but the in-link CSR is not built: ask the host
    L.done = done;
    for (int w = 0; w < kStWords; ++w)
        reinterpret_cast<unsigned long long *>(st)[w] = reinterpret_cast<const unsigned long long *>(&L)[w];
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
    if (threadIdx.x == 0) part[blockIdx.x].l1d = a;
}

// sum the partials in fixed order; a stop that the exact norm does not confirm resumes
__global__ void k_confirm(int G, int n, const ScanPartial *__restrict__ part, SolveState *__restrict__ st) {
    __shared__ double s[8];
    double a = 0.0;
    for (int c = threadIdx.x; c < G; c += blockDim.x) a += part[c].l1d;
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

// out[i] = src[new_of[i]] * scale, back in the caller's numbering; with partials the scale
// is 1/sum(partials) (the Section 3.3 renormalization H/|H|_1)
template <typename FT>
__global__ void k_gather_out(int n, const int *__restrict__ new_of, const FT *__restrict__ src,
                             const double *__restrict__ partials, int np, double *__restrict__ out) {
    __shared__ double scale;
    if (threadIdx.x == 0) {
        double a = 1.0;
        if (partials) {
            a = 0.0;
            for (int k = 0; k < np; ++k) a += partials[k];
            a = a > 0.0 ? 1.0 / a : 0.0;
        }
        scale = a;
    }
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)src[new_of[i]] * scale;
}


template <typename FT>
void launch_scan(di_graph *g, FT *F, const float *wsel, cudaStream_t s) {
    if (wsel)
        k_sweep_scan<FT, true><<<g->G, kScanThreads, 0, s>>>(g->chunk / kWarps, F, wsel, g->cls, g->region, g->W,
                                                             g->fcount, g->pre, sel_of<FT>(g), g->part,
                                                             g->st, g->H, rec_of<FT>(g), g->n, static_cast<FT *>(g->wpull));
    else
        k_sweep_scan<FT, false><<<g->G, kScanThreads, 0, s>>>(g->chunk / kWarps, F, nullptr, g->cls, g->region, g->W,
                                                              g->fcount, g->pre, sel_of<FT>(g), g->part,
                                                              g->st, g->H, rec_of<FT>(g), g->n, static_cast<FT *>(g->wpull));
}


int elem_grid(di_graph *g, long long work) {
    long long b = (work + 255) / 256;
    return (int)std::max(1LL, std::min(b, (long long)g->num_sms * 8));
}

// src (internal numbering) -> dst (caller's numbering, host or device)
template <typename FT>
di_status gather_out(di_graph *g, const FT *src, const double *partials, int np, double *dst, bool dst_dev) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    if (dst_dev) {
        k_gather_out<FT><<<elem_grid(g, n), 256, 0, s>>>(n, g->new_of, src, partials, np, dst);
        DI_CUDA(cudaGetLastError());
        return DI_OK;
    }
    double *tmp = nullptr;
    DI_CUDA(cudaMallocAsync(&tmp, sizeof(double) * (size_t)n, s));
    k_gather_out<FT><<<elem_grid(g, n), 256, 0, s>>>(n, g->new_of, src, partials, np, tmp);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(dst, tmp, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(tmp, s);
    return DI_OK;
}

// sweeps per iteration of the loop: its turn-around (a finalize's end to the next scan's start)
// took 5 us against 1.5 us between two kernels of the body (Zipf 2^24, globaltimer stamps), and
// four per iteration made the headline solve 1.7% faster than one
constexpr int kBodySweeps = 4;

// Build the while-loop graph of one precision: body = kBodySweeps x (scan -> push -> finalize).
template <typename FT>
di_status build_sweep_graph(di_graph *g, int slot, FT *F, const float *wsel) {
    di_status r = push_setup();
    if (r != DI_OK) return r;
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
    // kBodySweeps sweeps per loop iteration: the loop's turn-around costs more than a launch
    // inside the body; after the stop every kernel of the remaining sweeps returns at once
    for (int k = 0; k < kBodySweeps; ++k) {
        launch_scan<FT>(g, F, wsel, g->cap);
        launch_push<FT>(g, F, g->cap);
        if (slot >= kSweepSlots / 2) launch_pull<FT>(g, F, g->cap);  // returns at once on push sweeps
        k_sweep_finalize<<<1, 256, 0, g->cap>>>(g->n, g->G, g->part, g->st, g->trace, handle, 1);
    }
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

// how a solve starts: F_0 = (1-d)V, F_0 on the seeds of a query, or the state already in F and H
enum InitKind { kInitV, kInitSeeds, kInitState };

template <typename FT>
di_status solve_impl(di_graph *g, const di_solve_opts &o, FT *F, int slot, InitKind init, const int *seeds,
                     const double *seed_w, int nseeds, double wsum, double *H_out, bool out_dev, di_stats *stats) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    const int npad = g->G * g->chunk;
    const double omd = 1.0 - g->d;
    const float *wsel = o.select ? g->wsel[o.select - 1] : nullptr;
    const double wscale = o.select ? g->wscale[o.select - 1] : 1.0;
    // `slot` is the push-only loop; the loop with the pull kernel sits kSweepSlots/2 further on.
    // direction 2 before the in-link CSR exists runs push-only and pauses when a pull is due.
    bool pulls = o.direction == 1 || (o.direction == 2 && g->wpull != nullptr);
    const int pause_pull = o.direction == 2 && !pulls ? 1 : 0;
    if (pulls) slot += kSweepSlots / 2;
    if (!g->exec[slot]) {
        di_status r = build_sweep_graph<FT>(g, slot, F, wsel);
        if (r != DI_OK) return r;
    }
    // a graph update records ev0 itself, before its injection kernels
    if (init != kInitState) DI_CUDA(cudaEventRecord(g->ev0, s));
    if (init == kInitSeeds) {
        k_init_zero<FT><<<elem_grid(g, npad), 256, 0, s>>>(npad, n, F, g->H);
        k_init_seeds<FT><<<std::max(1, std::min(1024, (nseeds + 255) / 256)), 256, 0, s>>>(nseeds, seeds, seed_w, wsum,
                                                                                          omd, g->new_of, F);
    } else if (init == kInitV) {
        k_init_state<FT><<<elem_grid(g, npad), 256, 0, s>>>(n, npad, F, g->H, g->V, omd);
    }
    const double beta = o.beta > 0 ? o.beta : 0.5;
    const int max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 1000000;
    // a sweep that diffused at least half of all out-links is dense
    const long long pull_edges = o.direction ? std::max(1LL, (g->nnz + kPullShareSolve - 1) / kPullShareSolve)
                                             : std::numeric_limits<long long>::max();
    const int wait_polls = o.scan_wait_polls > 0 ? o.scan_wait_polls : kScanWaitLimit;
    if (init == kInitState) {
        k_l1_partials<FT><<<g->G, kScanThreads, 0, s>>>(n, g->chunk, F, g->part);
        k_init_control_l1<<<1, 32, 0, s>>>(g->st, g->part, g->G, o.tol * omd, beta, omd, n, o.max_edge_pushes,
                                           max_sweeps, o.trace ? 1 : 0, wscale, o.select ? 1 : 0, pull_edges, wait_polls,
                                           pause_pull);
    } else {
        k_init_control<<<1, 1, 0, s>>>(g->st, omd, o.tol * omd, beta, omd, n, o.max_edge_pushes, max_sweeps,
                                       o.trace ? 1 : 0, wscale, o.select ? 1 : 0, pull_edges, wait_polls, pause_pull);
    }
    DI_CUDA(cudaGetLastError());
    int attempts = 0;
    int pulling = 0;  // the device's pull flag before the next sweep (a profiled loop counts pull sweeps)
    g->prof = di_profile{};
    g->h_st->done = 0;  // the host copy of the previous solve's stop code is not this solve's
    for (int attempt = 0; attempt < 8; ++attempt) {
        ++attempts;
        if (g->h_st->done == 5) {
            // the loop paused for the in-link CSR: build it and the loop with the pull kernel,
            // then resume from the same state (this pause is not a confirmation attempt)
            di_status r = ensure_pull(g);
            if (r != DI_OK) return r;
            pulls = true;
            slot += kSweepSlots / 2;
            if (!g->exec[slot]) {
                r = build_sweep_graph<FT>(g, slot, F, wsel);
                if (r != DI_OK) return r;
            }
            k_resume_pull<<<1, 1, 0, s>>>(g->st);
            DI_CUDA(cudaGetLastError());
            --attempt;
        }
        if (o.profile) {
            // same kernels and arguments as the graph body, launched from the host with events around each
            cudaGraphConditionalHandle none = 0;
            for (;;) {
                DI_CUDA(cudaEventRecord(g->pev[0], s));
                launch_scan<FT>(g, F, wsel, s);
                DI_CUDA(cudaEventRecord(g->pev[1], s));
                launch_push<FT>(g, F, s);
                if (pulls) launch_pull<FT>(g, F, s);
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
                if (g->sweep_ms && g->prof.sweeps < kTraceCap) {
                    g->sweep_ms[2 * g->prof.sweeps] = t0;
                    g->sweep_ms[2 * g->prof.sweeps + 1] = t1;
                }
                g->prof.sweeps += 1;
                g->prof.pull_sweeps += pulls && pulling;
                pulling = g->h_st->pull;
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
        pulling = g->h_st->pull;
        if (g->h_st->done != 0 && g->h_st->done != 5) break;
    }
    DI_CUDA(cudaEventRecord(g->ev1, s));
    // outputs, in the caller's numbering
    if (H_out) {
        const int np = elem_grid(g, n);
        double *partials = nullptr;
        if (o.normalize) {
            DI_CUDA(cudaMallocAsync(&partials, sizeof(double) * (size_t)np, s));
            k_sum_h<<<np, 256, 0, s>>>(n, g->H, partials);
        }
        di_status r = gather_out<double>(g, g->H, partials, np, H_out, out_dev);
        if (partials) cudaFreeAsync(partials, s);
        if (r != DI_OK) return r;
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
        // init (2 kernels, 3 for a seeded query) + 3 per sweep of the loop (scan, push, finalize; 4
        // with the pull kernel), counting the sweeps of the last iteration that returned at once,
        // + 2 per confirmation
        stats->kernel_launches = (init == kInitV ? 2 : 3) + (pulls ? 4LL : 3LL) * h.body_runs + 2LL * attempts;
    }
#ifdef DI_DEBUG
    if (di_status dr = debug_status(); dr != DI_OK) return dr;
#endif
    if (h.done == 3) return set_error(DI_EKERNEL, "residual became non-finite");
    if (h.done == 4 && h.undrained) {
        g->untrusted = true;  // sticky: every later call on this graph fails until di_free
        return set_error(DI_ETIMEOUT, "a bulk-copy wait of the sweep scan gave up with copies still in flight; "
                                      "the graph must be freed");
    }
    if (h.done == 4) return set_error(DI_ETIMEOUT, "a bulk-copy wait of the sweep scan gave up");
    if (h.done != 1) return set_error(DI_ENOTCONVERGED, "stopped by a limit before |F|_1/(1-d) <= tol");
    return DI_OK;
}

}  // namespace

int scan_blocks_per_sm() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_sweep_scan<double, false>, kScanThreads, 0) != cudaSuccess)
        a = 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_scan<float, false>, kScanThreads, 0) != cudaSuccess)
        b = 4;
    cudaGetLastError();
    return std::max(1, std::min(a, b));
}

di_status sweep_alloc(di_graph *g) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    const int npad = g->G * g->chunk;
    DI_CUDA(cudaMallocAsync(&g->H, sizeof(double) * (size_t)npad, s));
    DI_CUDA(cudaMallocAsync(&g->sel, sizeof(Sel<double>) * (size_t)std::max(1, n), s));
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

namespace {

// ALGO-OP (select 1): w_i = 1/((#in_i + 1)(#out_i + 1)); ALGO-OP2 (select 2): w_i = 1/(#out_i + 1)
// (Section 4.3).  The integer product is converted to FP64, divided into 1 and rounded to FP32.
__global__ void k_sel_weights(int n, int npad, int select, const int *__restrict__ in_ptr,
                              const RowRec<double> *__restrict__ rec, float *__restrict__ w,
                              double *__restrict__ partial) {
    __shared__ double s_red[8];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < n) {
            const long long outd = rec[i].deg;
            const long long c = select == 1 ? (long long)(in_ptr[i + 1] - in_ptr[i] + 1) * (outd + 1) : outd + 1;
            v = __double2float_rn(1.0 / (double)c);
            acc += (double)v;
        }
        w[i] = v;
    }
    acc = block_sum(acc, s_red);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// the pull direction's inputs: the in-links with their targets, and the per-node pushed values
di_status ensure_pull(di_graph *g) {
    if (g->wpull) return DI_OK;
    di_status r = build_in_dst(g);
    if (r != DI_OK) return r;
    DI_CUDA(cudaMallocAsync(&g->wpull, sizeof(double) * (size_t)g->G * g->chunk, g->stream));
    return DI_OK;
}

di_status ensure_weights(di_graph *g, int select) {
    if (select == 0 || g->wsel[select - 1]) return DI_OK;
    di_status tr = build_transpose(g);  // #in_i
    if (tr != DI_OK) return tr;
    cudaStream_t s = g->stream;
    const int npad = g->G * g->chunk;
    float *w = nullptr;
    double *partial = nullptr;
    const int nb = elem_grid(g, npad);
    DI_CUDA(cudaMallocAsync(&w, sizeof(float) * (size_t)npad, s));
    DI_CUDA(cudaMallocAsync(&partial, sizeof(double) * (size_t)nb, s));
    k_sel_weights<<<nb, 256, 0, s>>>(g->n, npad, select, g->in_ptr, g->rec64, w, partial);
    DI_CUDA(cudaGetLastError());
    std::vector<double> h(nb);
    DI_CUDA(cudaMemcpyAsync(h.data(), partial, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(partial, s);
    double sum = 0.0;
    for (double x : h) sum += x;
    int ex = 0;
    std::frexp(sum / (double)g->n, &ex);            // mean = m 2^ex, 1/2 <= m < 1
    g->wscale[select - 1] = std::ldexp(1.0, ex - 1);  // 2^floor(log2(mean))
    g->wsel[select - 1] = w;
    return DI_OK;
}

// The updating equation (Section 3.2).  The old state, in the old graph's numbering,
// is moved to the new graph's numbering: r_new = new_of_new[perm_old[r_old]].
__global__ void k_map_state(int n, const int *__restrict__ perm_old, const int *__restrict__ new_of_new,
                            const double *__restrict__ F_old, const double *__restrict__ H_old,
                            double *__restrict__ F_new, double *__restrict__ H_new) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int t = new_of_new[perm_old[r]];
        F_new[t] = F_old[r];
        H_new[t] = H_old[r];
    }
}

// The injection F_0' = F + d(P' - P)H, row by row.  Rows whose fingerprints agree are the same
// in both graphs and cancel; a changed row of input node v takes back H_v d/#out_old along its
// old out-links (targets renumbered by old_to_new) and adds H_v d/#out_new along its new ones.
struct InjectArgs {
    int n;
    const unsigned long long *hash_old, *hash_new;
    const int *new_of_old, *new_of_new;
    const int *old_to_new;  // [n] old internal id -> new internal id
    const RowRec<double> *rec_old, *rec_new;
    const int *col_old, *col_new;
    const double *H;        // new numbering
    double *F;              // new numbering
    int *long_rows;         // changed rows with more than 32 out-links in either graph
    int *n_long;
    int n_hot;              // the new graph's hot targets (ids 0..n_hot-1), summed per CTA in shared memory
};

// one injected amount: the hot targets, which take a large share of all links and whose
// same-address reductions would serialize in one L2 slice, are summed in shared memory
__device__ __forceinline__ void inject_one(const InjectArgs &a, double *s_hot, int c, double val) {
    if (c < a.n_hot) atomicAdd(s_hot + c, val);
    else atomicAdd(a.F + c, val);
}

__device__ __forceinline__ void hot_zero(double *s_hot) {
    for (int k = threadIdx.x; k < kHotSlots; k += blockDim.x) s_hot[k] = 0.0;
    __syncthreads();
}

__device__ __forceinline__ void hot_flush(const InjectArgs &a, const double *s_hot) {
    __syncthreads();
    for (int k = threadIdx.x; k < a.n_hot; k += blockDim.x)
        if (s_hot[k] != 0.0) atomicAdd(a.F + k, s_hot[k]);
}

constexpr int kInjectRun = 4;

__device__ __forceinline__ void inject_row(const InjectArgs &a, double *s_hot, int v, int lane, int width) {
    const int ro = a.new_of_old[v], rn = a.new_of_new[v];
    const double h = a.H[rn];
    if (h == 0.0) return;
    const RowRec<double> o = a.rec_old[ro], w = a.rec_new[rn];
    const double vo = -h * o.inv, vn = h * w.inv;
    // kInjectRun out-links per thread and pass, their loads issued together: a long row is a
    // chain of dependent loads (column, renumbering) and reductions, bound by their latency
    constexpr int U = kInjectRun;
    for (int e0 = lane; e0 < o.deg; e0 += U * width) {
        int c[U];
#pragma unroll
        for (int k = 0; k < U; ++k) c[k] = e0 + k * width < o.deg ? a.col_old[o.beg + e0 + k * width] : -1;
#pragma unroll
        for (int k = 0; k < U; ++k) c[k] = c[k] >= 0 ? a.old_to_new[c[k]] : -1;
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c[k] >= 0) inject_one(a, s_hot, c[k], vo);
    }
    for (int e0 = lane; e0 < w.deg; e0 += U * width) {
        int c[U];
#pragma unroll
        for (int k = 0; k < U; ++k) c[k] = e0 + k * width < w.deg ? a.col_new[w.beg + e0 + k * width] : -1;
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c[k] >= 0) inject_one(a, s_hot, c[k], vn);
    }
}

__global__ void k_old_to_new(int n, const int *__restrict__ perm_old, const int *__restrict__ new_of_new,
                             int *__restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        out[r] = new_of_new[perm_old[r]];
}

// a thread per changed row of up to 32 out-links; longer ones are listed for k_inject_long
__global__ void k_inject_changed(InjectArgs a) {
    __shared__ double s_hot[kHotSlots];
    hot_zero(s_hot);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
        if (a.hash_old[v] == a.hash_new[v]) continue;
        const int dl = max(a.rec_old[a.new_of_old[v]].deg, a.rec_new[a.new_of_new[v]].deg);
        if (dl <= 32) inject_row(a, s_hot, v, 0, 1);
        else a.long_rows[atomicAdd(a.n_long, 1)] = v;
    }
    hot_flush(a, s_hot);
}

// a CTA per long changed row
__global__ void k_inject_long(InjectArgs a) {
    __shared__ double s_hot[kHotSlots];
    hot_zero(s_hot);
    const int cnt = *a.n_long;
    for (int k = blockIdx.x; k < cnt; k += gridDim.x) inject_row(a, s_hot, a.long_rows[k], threadIdx.x, blockDim.x);
    hot_flush(a, s_hot);
}

}  // namespace

#ifdef DI_DEBUG
namespace {
// records one failed check (code 99, index 12345) without touching memory
__global__ void k_dbg_selftest() {
    if (threadIdx.x == 0) (void)DI_CHECK(false, 99, 12345);
}
}  // namespace

unsigned long long dbg_take_sweep() { return dbg_take_word(); }

// the first failed index check of the sweep kernels (scan, push, pull) since the last call
di_status debug_status(unsigned long long *word) {
    unsigned long long w = dbg_take_sweep();
    const unsigned long long wp = dbg_take_push();
    if (!w) w = wp;
    if (word) *word = w;
    if (!w) return DI_OK;
    static const char *what[] = {"", "a scan list append beyond its warp's region",
                                 "a push list position beyond its sub-chunk's region", "a listed node id outside [0, n)",
                                 "a pushed-to column outside [0, n)", "a pull link endpoint outside [0, n)"};
    const unsigned code = (unsigned)(w >> 48);
    const long long idx = (long long)(w & 0xffffffffffffull);
    const char *msg = code < 6 ? what[code] : (code == 99 ? "the debug self-test" : "unknown check");
    return set_error(DI_EKERNEL, std::string("debug check ") + std::to_string(code) + " failed (" + msg +
                                     ") at index " + std::to_string(idx));
}

di_status debug_selftest(unsigned long long *word) {
    k_dbg_selftest<<<1, 32>>>();
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaDeviceSynchronize());
    return debug_status(word);
}
#endif

di_status selftest_wait(int polls, int ctas, int *gave_up) {
    int *d = nullptr;
    DI_CUDA(cudaMalloc(&d, sizeof(int)));
    cudaError_t e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_selftest_wait<<<ctas, 32>>>(polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(gave_up, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "di_selftest_wait");
    return DI_OK;
}

di_status run_solve(di_graph *g, const di_solve_opts &o, const int *seeds, const double *seed_w, int nseeds,
                    double wsum, double *H_out, bool out_dev, di_stats *st) {
    di_status r = ensure_fluid(g, o.prec);
    if (r != DI_OK) return r;
    r = ensure_weights(g, o.select);
    if (r != DI_OK) return r;
    g->last_prec = o.prec;
    g->last_trace_on = o.trace ? 1 : 0;
    if (o.direction == 1) {
        r = ensure_pull(g);
        if (r != DI_OK) return r;
    }
    const InitKind init = seeds ? kInitSeeds : kInitV;
    const int slot = o.select ? 3 + 2 * (o.select - 1) + o.prec : o.prec;  // the push-only loop
    if (o.prec == DI_FP64)
        return solve_impl<double>(g, o, g->F64, slot, init, seeds, seed_w, nseeds, wsum, H_out, out_dev, st);
    return solve_impl<float>(g, o, g->F32, slot, init, seeds, seed_w, nseeds, wsum, H_out, out_dev, st);
}

di_status run_update(di_graph *go, di_graph *gn, const di_solve_opts &o, double *H_out, bool out_dev, di_stats *st) {
    di_status r = ensure_fluid(gn, DI_FP64);
    if (r != DI_OK) return r;
    r = ensure_weights(gn, o.select);
    if (r != DI_OK) return r;
    if (o.direction == 1) {
        r = ensure_pull(gn);
        if (r != DI_OK) return r;
    }
    const int n = gn->n;
    const int slot = o.select ? 3 + 2 * (o.select - 1) : 0;  // the push-only loop
    const bool pulls = o.direction == 1 || (o.direction == 2 && gn->wpull != nullptr);
    const int cslot = slot + (pulls ? kSweepSlots / 2 : 0);
    if (!gn->exec[cslot]) {  // capture before timing starts, as a solve does
        r = build_sweep_graph<double>(gn, cslot, gn->F64, o.select ? gn->wsel[o.select - 1] : nullptr);
        if (r != DI_OK) return r;
    }
    if (go != gn) {  // the row fingerprints that find the changed rows, at the first update
        r = ensure_rowhash(go);
        if (r == DI_OK) r = ensure_rowhash(gn);
        if (r != DI_OK) return r;
    }
    // both graphs' earlier work is complete before the new graph's stream reads the old state
    DI_CUDA(cudaStreamSynchronize(go->stream));
    DI_CUDA(cudaEventRecord(gn->ev0, gn->stream));
    if (go != gn) {
        cudaStream_t s = gn->stream;
        const int npad = gn->G * gn->chunk;
        // the state in the new numbering, then F_0' = F + d(P' - P)H over the changed rows only
        DI_CUDA(cudaMemsetAsync(gn->F64, 0, sizeof(double) * (size_t)npad, s));
        DI_CUDA(cudaMemsetAsync(gn->H, 0, sizeof(double) * (size_t)npad, s));
        k_map_state<<<elem_grid(gn, n), 256, 0, s>>>(n, go->perm, gn->new_of, go->F64, go->H, gn->F64, gn->H);
        InjectArgs a;
        a.n = n;
        a.hash_old = go->rowhash;
        a.hash_new = gn->rowhash;
        a.new_of_old = go->new_of;
        a.new_of_new = gn->new_of;
        a.rec_old = go->rec64;
        a.rec_new = gn->rec64;
        a.col_old = go->col_idx;
        a.col_new = gn->col_idx;
        a.H = gn->H;
        a.F = gn->F64;
        a.n_hot = std::min(gn->n_hot, kHotSlots);
        // scratch: the composed renumbering, the long-row list (at most L/33 rows of either
        // graph have more than 32 out-links) and its count
        const long long cap = (go->nnz + gn->nnz) / 33 + 1;
        int *o2n = nullptr, *lrows = nullptr, *cnt = nullptr;
        DI_CUDA(cudaMallocAsync(&o2n, sizeof(int) * (size_t)n, s));
        DI_CUDA(cudaMallocAsync(&lrows, sizeof(int) * (size_t)cap, s));
        DI_CUDA(cudaMallocAsync(&cnt, sizeof(int), s));
        DI_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
        a.old_to_new = o2n;
        a.long_rows = lrows;
        a.n_long = cnt;
        k_old_to_new<<<elem_grid(gn, n), 256, 0, s>>>(n, go->perm, gn->new_of, o2n);
        k_inject_changed<<<elem_grid(gn, n), 256, 0, s>>>(a);
        k_inject_long<<<gn->num_sms * 4, 256, 0, s>>>(a);
        DI_CUDA(cudaGetLastError());
        cudaFreeAsync(o2n, s);
        cudaFreeAsync(lrows, s);
        cudaFreeAsync(cnt, s);
    }
    gn->last_prec = DI_FP64;
    gn->last_trace_on = o.trace ? 1 : 0;
    return solve_impl<double>(gn, o, gn->F64, slot, kInitState, nullptr, nullptr, 0, 1.0, H_out, out_dev, st);
}

di_status gather_x(di_graph *g, const double *src, double *dst, bool dst_dev) {
    return gather_out<double>(g, src, nullptr, 0, dst, dst_dev);
}

di_status copy_state(const di_graph *gc, double *F_out, bool F_dev, double *H_out, bool H_dev) {
    di_graph *g = const_cast<di_graph *>(gc);
    if (F_out) {
        di_status r;
        if (g->last_prec == DI_FP32_MIXED && g->F32) r = gather_out<float>(g, g->F32, nullptr, 0, F_out, F_dev);
        else if (g->F64) r = gather_out<double>(g, g->F64, nullptr, 0, F_out, F_dev);
        else return set_error(DI_EINVAL, "no solve has run on this graph");
        if (r != DI_OK) return r;
    }
    if (H_out) {
        di_status r = gather_out<double>(g, g->H, nullptr, 0, H_out, H_dev);
        if (r != DI_OK) return r;
    }
    DI_CUDA(cudaStreamSynchronize(g->stream));
    return DI_OK;
}

namespace {

// a saved state in the caller's numbering, moved into the internal one; flags non-finite values
__global__ void k_state_in(int n, const int *__restrict__ perm, const double *__restrict__ F_in,
                           const double *__restrict__ H_in, double *__restrict__ F, double *__restrict__ H,
                           int *__restrict__ bad) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const double f = F_in[perm[r]], h = H_in[perm[r]];
        if (!isfinite(f) || !isfinite(h)) atomicOr(bad, 1);
        F[r] = f;
        H[r] = h;
    }
}

// Theorem 1 residual, first part: Z = F_0 - H - F with F_0 = (1-d)V
__global__ void k_state_z(int n, double omd, const double *__restrict__ V, const double *__restrict__ F,
                          const double *__restrict__ H, double *__restrict__ Z) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        Z[r] = omd * (V ? V[r] : 1.0 / (double)n) - H[r] - F[r];
}

// then Z += dPH: a warp per row i adds d*H_i/#out_i to every child
__global__ void k_state_dph(int n, const RowRec<double> *__restrict__ rec, const int *__restrict__ col_idx,
                            const double *__restrict__ H, double *__restrict__ Z) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const RowRec<double> rr = rec[i];
        const double w = H[i] * rr.inv;
        if (w == 0.0) continue;
        for (int k = lane; k < rr.deg; k += 32) atomicAdd(Z + col_idx[rr.beg + k], w);
    }
}

// max_j |Z_j| and max_j (|H_j| + |F_j| + (1-d)V_j), as non-negative doubles ordered by their bits
__global__ void k_state_max(int n, double omd, const double *__restrict__ V, const double *__restrict__ F,
                            const double *__restrict__ H, const double *__restrict__ Z,
                            unsigned long long *__restrict__ out) {
    double zm = 0.0, sm = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        zm = fmax(zm, fabs(Z[r]));
        sm = fmax(sm, fabs(H[r]) + fabs(F[r]) + omd * (V ? V[r] : 1.0 / (double)n));
    }
    for (int o = 16; o > 0; o >>= 1) {
        zm = fmax(zm, __shfl_down_sync(kFull, zm, o));
        sm = fmax(sm, __shfl_down_sync(kFull, sm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(zm));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(sm));
    }
}

}  // namespace

di_status set_state(di_graph *g, const double *F_in, bool F_dev, const double *H_in, bool H_dev, double rtol,
                    double *deviation) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    const int npad = g->G * g->chunk;
    di_status r = ensure_fluid(g, DI_FP64);
    if (r != DI_OK) return r;
    double *bufs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // F_in, H_in copies, F, H, Z
    int *bad = nullptr;
    unsigned long long *mx = nullptr;
    auto release = [&]() {
        for (double *b : bufs)
            if (b) cudaFreeAsync(b, s);
        if (bad) cudaFreeAsync(bad, s);
        if (mx) cudaFreeAsync(mx, s);
        cudaStreamSynchronize(s);
    };
    const size_t bytes = sizeof(double) * (size_t)n;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
        if ((k == 0 && F_dev) || (k == 1 && H_dev)) continue;
        e = cudaMallocAsync(&bufs[k], k >= 2 ? sizeof(double) * (size_t)npad : bytes, s);
    }
    if (e == cudaSuccess) e = cudaMallocAsync(&bad, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&mx, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), s);
    const double *Fs = F_in, *Hs = H_in;
    if (e == cudaSuccess && !F_dev) {
        e = cudaMemcpyAsync(bufs[0], F_in, bytes, cudaMemcpyHostToDevice, s);
        Fs = bufs[0];
    }
    if (e == cudaSuccess && !H_dev) {
        e = cudaMemcpyAsync(bufs[1], H_in, bytes, cudaMemcpyHostToDevice, s);
        Hs = bufs[1];
    }
    double *F = bufs[2], *H = bufs[3], *Z = bufs[4];
    if (e == cudaSuccess) e = cudaMemsetAsync(F, 0, sizeof(double) * (size_t)npad, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(H, 0, sizeof(double) * (size_t)npad, s);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "state upload");
    }
    const int grid = elem_grid(g, n);
    k_state_in<<<grid, 256, 0, s>>>(n, g->perm, Fs, Hs, F, H, bad);
    k_state_z<<<grid, 256, 0, s>>>(n, 1.0 - g->d, g->V, F, H, Z);
    k_state_dph<<<g->num_sms * 8, 256, 0, s>>>(n, g->rec64, g->col_idx, H, Z);
    k_state_max<<<grid, 256, 0, s>>>(n, 1.0 - g->d, g->V, F, H, Z, mx);
    e = cudaGetLastError();
    int hbad = 0;
    unsigned long long hm[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "state check");
    }
    if (hbad) {
        release();
        return set_error(DI_EINVAL, "di_set_state: F or H holds a NaN or an infinity");
    }
    double zmax, scale;
    std::memcpy(&zmax, &hm[0], sizeof(double));
    std::memcpy(&scale, &hm[1], sizeof(double));
    const double dev = scale > 0.0 ? zmax / scale : zmax;
    if (deviation) *deviation = dev;
    if (!(dev <= rtol)) {
        release();
        return set_error(DI_EINVAL, "di_set_state: the state breaks Theorem 1 (H + F = (1-d)V + dPH): relative "
                                    "deviation " + std::to_string(dev) + " > rtol " + std::to_string(rtol));
    }
    // accepted: the graph's FP64 state becomes (F, H), as if its last solve had stopped there
    e = cudaMemcpyAsync(g->F64, F, sizeof(double) * (size_t)npad, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->H, H, sizeof(double) * (size_t)npad, cudaMemcpyDeviceToDevice, s);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "state load");
    g->last_prec = DI_FP64;
    g->last_trace_on = 0;
    return DI_OK;
}

}  // namespace diter
