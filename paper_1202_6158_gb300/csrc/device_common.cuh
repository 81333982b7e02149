// device_common.cuh -- device helpers shared by the sweep kernels (single and batched).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace diter {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Fire-and-forget reductions into F (performed by the L2 atomic units).  No memory
// clobber: nothing in a push kernel reads F, so loads may be scheduled freely
// around these.
__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void red_add(float *p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v));
}
// the same with an L2 eviction policy (evict_last keeps the updated lines of F and H in L2)
__device__ __forceinline__ void red_add(double *p, double v, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol));
}
__device__ __forceinline__ void red_add(float *p, float v, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol));
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

// Streaming loads of the scan carry an L2 evict-first policy so that the scan's
// pass over all of F does not push the push kernel's working set out of L2.  (F is
// written by the scan itself, so its loads stay on the coherent path; the class
// bytes are read-only.)
// ---- bulk copies (TMA, 1-D) into shared memory, completed on an mbarrier
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// global -> shared, bytes a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy(unsigned dst, const void *src, unsigned bytes, unsigned bar,
                                          unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(pol) : "memory");
}

// one bounded wait for the given phase: false if it did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase, int limit) {
    for (int it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long evict_last_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long evict_first_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double2 ld_stream(const double2 *a, unsigned long long pol) {
    double2 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4 *a, unsigned long long pol) {
    float4 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned ld_stream(const unsigned *a, unsigned long long pol) {
    unsigned v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

// The last batched-scan CTA to finish (a ticket counter, no waiting) turns the per-sub-chunk
// counts into exclusive prefix sums per list, so the push can spread the selected
// nodes evenly over all its warps whatever their distribution over the chunks.
// Each thread sums a contiguous run of sub-chunks for every list, one block scan
// covers the four lists, then each thread writes its run.  (prefix_counts below uses the
// CTA-parallel pass when its staging buffer holds the CTA sums.)
// s_c: kCap ints of shared memory to stage the counts in
// rows first_list..kCountRows-1: the lists, then the hub chunk counts (the others are left as they are)
__device__ void prefix_counts_staged(const int *__restrict__ fcount, int W, int *__restrict__ pre, int *s_c,
                                     const int kCap, int first_list = 0) {
    __shared__ int s_w[kWarps];
    __shared__ int s_carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int L = first_list; L < kCountRows; ++L) {
        if (threadIdx.x == 0) s_carry = 0;
        for (int base = 0; base < W; base += kCap) {
            const int m = min(kCap, W - base);
            // coalesced loads, all in flight together
            for (int t = threadIdx.x; t < m; t += kScanThreads) s_c[t] = __ldcg(fcount + L * W + base + t);
            __syncthreads();
            const int per = (m + kScanThreads - 1) / kScanThreads;
            const int g0 = min(m, threadIdx.x * per), g1 = min(m, g0 + per);
            int a = 0;
            for (int g = g0; g < g1; ++g) a += s_c[g];
            int x = a;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_w[w] = x;
            __syncthreads();
            int off = s_carry, tot = 0;
            for (int k = 0; k < kWarps; ++k) {
                off += k < w ? s_w[k] : 0;
                tot += s_w[k];
            }
            int run = off + x - a;
            for (int g = g0; g < g1; ++g) {
                pre[L * (W + 1) + base + g] = run;
                run += s_c[g];
            }
            __syncthreads();
            if (threadIdx.x == 0) s_carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) pre[L * (W + 1) + W] = s_carry;
        __syncthreads();
    }
}

// The same prefix sums with the work spread over the CTA (W = G * kWarps, the counts of one
// scan CTA's eight warps adjacent): thread t takes the scan CTAs t, t + 256, ...; two 16-byte
// loads per CTA and row give its eight counts, whose sum goes to s_tot; one warp per row scans
// the CTA sums in place; the same thread then writes the CTA's eight offsets.  s_tot holds
// (kCountRows - first_list) * G ints.
__device__ void prefix_counts_by_cta(const int *__restrict__ fcount, int G, int W, int *__restrict__ pre, int *s_tot,
                                     int first_list) {
    __shared__ int s_rowtot[kCountRows];
    const int R = kCountRows - first_list;
    for (int b = threadIdx.x; b < G; b += kScanThreads) {
        for (int r = 0; r < R; ++r) {
            const int4 *p = reinterpret_cast<const int4 *>(fcount + (first_list + r) * W + b * kWarps);
            const int4 x = __ldcg(p), y = __ldcg(p + 1);
            s_tot[r * G + b] = x.x + x.y + x.z + x.w + y.x + y.y + y.z + y.w;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < R) {  // warp w: exclusive scan of row w's CTA sums, in place
        int *t = s_tot + w * G;
        const int per = (G + 31) / 32, b0 = min(G, lane * per), b1 = min(G, b0 + per);
        int a = 0;
        for (int b = b0; b < b1; ++b) a += t[b];
        int x = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_rowtot[w] = x;
        int run = x - a;
        for (int b = b0; b < b1; ++b) {
            const int c = t[b];
            t[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < G; b += kScanThreads) {
        for (int r = 0; r < R; ++r) {
            const int L = first_list + r;
            const int4 *p = reinterpret_cast<const int4 *>(fcount + L * W + b * kWarps);
            const int4 x = __ldcg(p), y = __ldcg(p + 1);
            const int c[kWarps] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
            int *o = pre + L * (W + 1) + b * kWarps;
            int run = s_tot[r * G + b];
#pragma unroll
            for (int k = 0; k < kWarps; ++k) {
                o[k] = run;
                run += c[k];
            }
        }
    }
    if ((int)threadIdx.x < R) pre[(first_list + threadIdx.x) * (W + 1) + W] = s_rowtot[threadIdx.x];
    __syncthreads();
}
static_assert(kWarps == 8, "a CTA's counts of a row are read as two int4");

// called by the last CTA of a scan grid of G = W / kWarps CTAs
__device__ void prefix_counts(const int *__restrict__ fcount, int W, int *__restrict__ pre, int first_list = 0) {
    constexpr int kCap = 8192;                     // sub-chunks staged per pass (32 KB)
    __shared__ int s_c[kCap];
    const int G = W / kWarps;
    if ((kCountRows - first_list) * G <= kCap && (int)gridDim.x == G)
        prefix_counts_by_cta(fcount, G, W, pre, s_c, first_list);
    else
        prefix_counts_staged(fcount, W, pre, s_c, kCap, first_list);
}

// sub-chunk holding item t of a list: the last g with pre[g] <= t
__device__ __forceinline__ int find_sub(const int *__restrict__ pre, int W, int t) {
    int lo = 0, hi = W;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// the same, knowing the answer is at least lo: a few steps forward, then a binary search
__device__ __forceinline__ int find_sub_from(const int *__restrict__ pre, int W, int t, int lo) {
    for (int k = 0; k < 4; ++k) {
        if (__ldg(pre + lo + 1) > t) return lo;
        ++lo;
    }
    int hi = W;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace
}  // namespace diter
