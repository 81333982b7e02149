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

// Fire-and-forget reductions into F (performed by the L2 atomic units).  No memory
// clobber: nothing in a push kernel reads F, so loads may be scheduled freely
// around these.
__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void red_add(float *p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v));
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

// FP64 fluid: the threshold test compares bit patterns as signed integers, which
// orders non-negative doubles exactly like their values (F >= 0 throughout).
template <>
struct ScanOps<double> {
    using VT = double2;
    static constexpr int VN = 2;
    using Key = long long;
    __device__ static Key key(double T) { return __double_as_longlong(T); }
    __device__ static bool above(double f, Key k) { return __double_as_longlong(f) > k; }
};

template <>
struct ScanOps<float> {
    using VT = float4;
    static constexpr int VN = 4;
    using Key = float;
    __device__ static Key key(double T) { return (float)T; }
    __device__ static bool above(float f, Key k) { return f > k; }
};

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_sweep_scan(int n, int chunk, FT *__restrict__ F,
                                                             double *__restrict__ H, const int *__restrict__ row_ptr,
                                                             const FT *__restrict__ inv_deg,
                                                             const int *__restrict__ region, int G,
                                                             int *__restrict__ fcount, FEntryT<FT> *__restrict__ frontier,
                                                             ScanPartial *__restrict__ part,
                                                             const SolveState *__restrict__ st, double d) {
    using Ops = ScanOps<FT>;
    using VT = typename Ops::VT;
    constexpr int VN = Ops::VN;
    constexpr int NW = kScanThreads / 32;
    __shared__ int s_wcnt[3][NW];
    __shared__ double s_red_d[NW];
    __shared__ long long s_red_l[NW];
    if (st->done) return;
    const typename Ops::Key key = Ops::key(st->T);
    const int S = fixed_scale(st->R);
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long beg = (long long)c * chunk;
    const long long end = min((long long)n, beg + chunk);
    int run0 = region[0 * (G + 1) + c], run1 = region[1 * (G + 1) + c], run2 = region[2 * (G + 1) + c];
    const int start0 = run0, start1 = run1, start2 = run2;
    long long l1 = 0;                 // |F|_1 over this thread's elements (fixed point)
    long long sent_out = 0, sent_dng = 0;  // fluid moved by selected nodes with / without children
    int edges = 0, srcs = 0, entries = 0;

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
        FEntryT<FT> ent[VN];
        bool any = false;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            const long long i = i0 + k;
            const FT fv = f[k];
            const long long fx = to_fixed(fv, S);
            l1 += fx;
            bin[k] = -1;
            if (i < end && Ops::above(fv, key)) {
                any = true;
                srcs += 1;
                H[i] += (double)fv;                 // J_i F: the fluid moves into the history
                f[k] = (FT)0;
                const int rb = row_ptr[i];
                const int deg = row_ptr[i + 1] - rb;
                if (deg == 0) {
                    sent_dng += fx;                 // a dangling node's fluid leaves (Section 3.3)
                } else {
                    sent_out += fx;
                    edges += deg;
                    entries += 1;
                    bin[k] = deg <= kOutCut1 ? 0 : (deg <= kOutCut2 ? 1 : 2);
                    ent[k].beg = rb;
                    ent[k].deg = deg;
                    ent[k].w = fv * inv_deg[i];     // d * sent / outdeg(i)
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
    (void)s_red_d;
    const long long bl1 = block_sum(l1, s_red_l);
    const long long bout = block_sum(sent_out, s_red_l);
    const long long bdng = block_sum(sent_dng, s_red_l);
    const long long bed = block_sum((long long)edges, s_red_l);
    const long long bsr = block_sum((long long)srcs, s_red_l);
    const long long ben = block_sum((long long)entries, s_red_l);
    if (threadIdx.x == 0) {
        ScanPartial p;
        p.l1 = bl1;
        p.out = bout;
        p.dng = bdng;
        p.edges = bed;
        p.srcs = bsr;
        p.entries = ben;
        p.l1d = 0.0;
        p.pad = 0.0;
        part[c] = p;
    }
}

// ------------------------------------------------------------------- push

// One elementary step F_j += w.  Edges into the hot targets (the most-linked-to
// nodes, encoded as -1 - slot) are summed in the CTA's shared memory: on power-law
// graphs a single target can receive a few percent of all pushes, and same-address
// reductions serialize in one L2 slice.
template <typename FT>
__device__ __forceinline__ void push_one(FT *__restrict__ F, FT *hot, int c, FT w) {
    if (c >= 0) red_add(F + c, w);
    else atomicAdd(hot + (-1 - c), w);
}

// Rows of the warp and CTA bins: the head up to a 16-byte boundary, then int4
// loads two at a time (all loads of a step are issued before its reductions),
// then the tail.
template <typename FT>
__device__ __forceinline__ void push_row_lanes(const int *__restrict__ col_idx, FT *__restrict__ F, FT *hot, int beg,
                                               int deg, FT w, int lane, int width) {
    const int head = min(deg, (4 - (beg & 3)) & 3);
    if (lane < head) push_one(F, hot, __ldg(col_idx + beg + lane), w);
    const int body = (deg - head) >> 2;
    const int4 *v4 = reinterpret_cast<const int4 *>(col_idx + beg + head);
    int k = lane;
    for (; k + width < body; k += 2 * width) {
        const int4 q = __ldg(v4 + k);
        const int4 r = __ldg(v4 + k + width);
        push_one(F, hot, q.x, w);
        push_one(F, hot, q.y, w);
        push_one(F, hot, q.z, w);
        push_one(F, hot, q.w, w);
        push_one(F, hot, r.x, w);
        push_one(F, hot, r.y, w);
        push_one(F, hot, r.z, w);
        push_one(F, hot, r.w, w);
    }
    if (k < body) {
        const int4 q = __ldg(v4 + k);
        push_one(F, hot, q.x, w);
        push_one(F, hot, q.y, w);
        push_one(F, hot, q.z, w);
        push_one(F, hot, q.w, w);
    }
    const int t = head + 4 * body + lane;
    if (t < deg) push_one(F, hot, __ldg(col_idx + beg + t), w);
}

// a thread-bin row (1..kOutCut1 out-links): all index loads first, then the reductions
template <typename FT>
__device__ __forceinline__ void push_short_row(const int *__restrict__ col_idx, FT *__restrict__ F, FT *hot,
                                               const FEntryT<FT> &e) {
    int c[kOutCut1];
#pragma unroll
    for (int t = 0; t < kOutCut1; ++t) c[t] = t < e.deg ? __ldg(col_idx + e.beg + t) : 0;
#pragma unroll
    for (int t = 0; t < kOutCut1; ++t)
        if (t < e.deg) push_one(F, hot, c[t], e.w);
}

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_sweep_push(const int *__restrict__ col_idx, FT *__restrict__ F,
                                                             const int *__restrict__ region,
                                                             const int *__restrict__ fcount, int G,
                                                             const FEntryT<FT> *__restrict__ frontier,
                                                             const int *__restrict__ hot_ids, int n_hot,
                                                             const SolveState *__restrict__ st) {
    __shared__ FT hot[kHotSlots];
    if (st->done) return;
    for (int t = threadIdx.x; t < kHotSlots; t += kScanThreads) hot[t] = (FT)0;
    __syncthreads();
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // CTA per source: the largest out-degrees
    {
        const int base = region[2 * (G + 1) + c], cnt = fcount[2 * G + c];
        for (int k = 0; k < cnt; ++k) {
            const FEntryT<FT> e = frontier[base + k];
            push_row_lanes(col_idx, F, hot, e.beg, e.deg, e.w, threadIdx.x, kScanThreads);
        }
    }
    // warp per source
    {
        const int base = region[1 * (G + 1) + c], cnt = fcount[1 * G + c];
        for (int k = w; k < cnt; k += kScanThreads / 32) {
            const FEntryT<FT> e = frontier[base + k];
            push_row_lanes(col_idx, F, hot, e.beg, e.deg, e.w, lane, 32);
        }
    }
    // thread per source, two sources in flight per thread
    {
        const int base = region[0 * (G + 1) + c], cnt = fcount[0 * G + c];
        int k = threadIdx.x;
        for (; k + kScanThreads < cnt; k += 2 * kScanThreads) {
            const FEntryT<FT> e0 = frontier[base + k];
            const FEntryT<FT> e1 = frontier[base + k + kScanThreads];
            push_short_row(col_idx, F, hot, e0);
            push_short_row(col_idx, F, hot, e1);
        }
        if (k < cnt) push_short_row(col_idx, F, hot, frontier[base + k]);
    }
    // the CTA's sums for the hot targets go to F once
    __syncthreads();
    for (int t = threadIdx.x; t < n_hot; t += kScanThreads) {
        const FT v = hot[t];
        if (v != (FT)0) red_add(F + hot_ids[t], v);
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
    (void)s_d;
    long long fl1 = 0, fout = 0, fdng = 0, ed = 0, sr = 0, en = 0;
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
        fl1 += part[c].l1;
        fout += part[c].out;
        fdng += part[c].dng;
        ed += part[c].edges;
        sr += part[c].srcs;
        en += part[c].entries;
    }
    fl1 = block_sum(fl1, s_l);
    fout = block_sum(fout, s_l);
    fdng = block_sum(fdng, s_l);
    ed = block_sum(ed, s_l);
    sr = block_sum(sr, s_l);
    en = block_sum(en, s_l);
    if (threadIdx.x != 0) return;
    st->body_runs += 1;
    const double Tused = st->T;
    const int S = fixed_scale(st->R);  // the scale the scan used (st->R is still the previous residual)
    const double l1 = ldexp((double)fl1, -S);
    // removed mass: (1-d)*sent for nodes with children, sent for dangling nodes (Section 3.3)
    const double rem = st->one_minus_d * ldexp((double)fout, -S) + ldexp((double)fdng, -S);
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
        r.scan_ms = 0.0;
        r.push_ms = 0.0;
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

template <typename FT> const FT *inv_deg_of(di_graph *g);
template <> const double *inv_deg_of<double>(di_graph *g) { return g->inv_deg; }
template <> const float *inv_deg_of<float>(di_graph *g) { return g->inv_deg32; }
template <typename FT> FEntryT<FT> *frontier_of(di_graph *g) { return reinterpret_cast<FEntryT<FT> *>(g->frontier); }

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
    k_sweep_scan<FT><<<g->G, kScanThreads, 0, g->cap>>>(g->n, g->chunk, F, g->H, g->row_ptr, inv_deg_of<FT>(g), g->region,
                                                         g->G, g->fcount, frontier_of<FT>(g), g->part, g->st, g->d);
    k_sweep_push<FT><<<g->G, kScanThreads, 0, g->cap>>>(g->col_idx, F, g->region, g->fcount, g->G, frontier_of<FT>(g),
                                                         g->hot_ids, g->n_hot, g->st);
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
                k_sweep_scan<FT><<<g->G, kScanThreads, 0, s>>>(n, g->chunk, F, g->H, g->row_ptr, inv_deg_of<FT>(g),
                                                              g->region, g->G, g->fcount, frontier_of<FT>(g), g->part,
                                                              g->st, g->d);
                DI_CUDA(cudaEventRecord(g->pev[1], s));
                k_sweep_push<FT><<<g->G, kScanThreads, 0, s>>>(g->col_idx, F, g->region, g->fcount, g->G,
                                                              frontier_of<FT>(g), g->hot_ids, g->n_hot, g->st);
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

int scan_blocks_per_sm() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_sweep_scan<double>, kScanThreads, 0) != cudaSuccess) a = 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_scan<float>, kScanThreads, 0) != cudaSuccess) b = 4;
    cudaGetLastError();
    return std::max(1, std::min(a, b));
}

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
