// graph_build.cu -- graph ingest on the device (create time).
//
// Everything the solves need is derived here by our own kernels, from the
// out-link CSR of the problem statement (Section 2.1: column j of P spreads
// 1/outdeg(j) over the children of j; Section 3.3: dangling columns stay zero):
//   * validation of the CSR and of V (error flags, no traps);
//   * the internal numbering (the most-linked-to targets first, every other node
//     in input order) and the CSR relabeled to it;
//   * out-degree bins (0 dangling, 1 thread, 2 warp, 3 CTA), the packed row
//     records and, per sweep-scan chunk, the offsets at which each bin's
//     selected nodes are written;
//   * at first use: the in-link CSR (a stable LSD radix sort of (target, source)
//     pairs, so every in-row lists its sources in ascending order and the result
//     is unique, hence bit-exact against any correct construction), the target of
//     each in-link, in-degree classes (exports) and row fingerprints (updates).
#include <cuda_runtime.h>

#include <climits>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace diter {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// exclusive scan of one int per thread over a 256-thread block; *total gets the block sum
__device__ int block_excl_scan(int v, int *total) {
    __shared__ int ws[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < 8 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < 8) ws[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (w > 0 ? ws[w - 1] : 0);
    *total = ws[7];
    __syncthreads();
    return excl;
}

// ---------------------------------------------------------------- validation

enum : int { kBadRowPtr0 = 1, kBadRowPtrN = 2, kNotMonotone = 4, kColRange = 8, kVNeg = 16, kVNonFinite = 32 };

// row starts; the column range is checked by the in-degree count that reads every column
__global__ void k_validate_rows(int n, long long nnz, const int *__restrict__ row_ptr, int *flags) {
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    int f = 0;
    if (tid == 0) {
        if (row_ptr[0] != 0) f |= kBadRowPtr0;
        if ((long long)row_ptr[n] != nnz) f |= kBadRowPtrN;
    }
    for (long long i = tid; i < n; i += stride)
        if (row_ptr[i + 1] < row_ptr[i]) f |= kNotMonotone;
    if (f) atomicOr(flags, f);
}

__global__ void k_validate_v(int n, const double *__restrict__ V, int *flags, double *sum) {
    double s = 0.0;
    int f = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = V[i];
        if (!isfinite(v)) f |= kVNonFinite;
        else if (v < 0.0) f |= kVNeg;
        else s += v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, s);
    if (f) atomicOr(flags, f);
}

// ------------------------------------------------------- degrees and bins

// out-degree class and d/outdeg of every node (the one division per node the solves need),
// and the packed row record {start, outdeg, d/outdeg} the push reads with one access
// d/k for k < kInvTable (0 for k = 0): FP64 division is scarce on this GPU (about 59 G/s), and a
// graph's out-degrees repeat, so each distinct small degree is divided once
constexpr int kInvTable = 1 << 16;
__global__ void k_inv_table(double d, double *__restrict__ tab) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kInvTable; k += gridDim.x * blockDim.x)
        tab[k] = k ? d / (double)k : 0.0;
}

__global__ void k_out_bins(int n, const int *__restrict__ row_ptr, int cut1, int cut2, double d,
                           const double *__restrict__ inv_tab, int *__restrict__ bin_of,
                           unsigned char *__restrict__ cls, double *__restrict__ inv_deg, float *__restrict__ inv_deg32,
                           RowRec<double> *__restrict__ rec64, RowRec<float> *__restrict__ rec32) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int beg = row_ptr[i];
        const int deg = row_ptr[i + 1] - beg;
        int b = deg == 0 ? 0 : (deg <= cut1 ? 1 : (deg <= cut2 ? 2 : 3));
        bin_of[i] = b;
        cls[i] = (unsigned char)(b < 3 ? b : 2 + hub_chunk_count(deg));
        // the same correctly rounded d/deg either way
        const double w = deg < kInvTable ? __ldg(inv_tab + deg) : d / (double)deg;
        inv_deg[i] = w;
        inv_deg32[i] = (float)w;
        RowRec<double> r64;
        r64.beg = beg;
        r64.deg = deg;
        r64.inv = w;
        rec64[i] = r64;
        RowRec<float> r32;
        r32.beg = beg;
        r32.deg = deg;
        r32.inv = (float)w;
        rec32[i] = r32;
    }
}

// per warp sub-chunk: how many nodes of each class it holds
__global__ void k_sub_counts(int n, int wchunk, const unsigned char *__restrict__ cls, int *__restrict__ cnt, int W) {
    __shared__ int c[kLists];
    if (threadIdx.x < kLists) c[threadIdx.x] = 0;
    __syncthreads();
    const long long beg = (long long)blockIdx.x * wchunk, end = min((long long)n, beg + wchunk);
    int l[kLists] = {0, 0, 0, 0};
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) l[class_of_byte(cls[i])] += 1;
    for (int L = 0; L < kLists; ++L) atomicAdd(&c[L], l[L]);
    __syncthreads();
    if (threadIdx.x < kLists) cnt[threadIdx.x * W + blockIdx.x] = c[threadIdx.x];
}

// region[L][g] = (nodes of classes < L) + (nodes of class L in sub-chunks < g), from the
// exclusive scan x of the flattened counts [kLists * W + 1]: region[L][g] = x[L*W + g]
__global__ void k_region_layout(int W, const int *__restrict__ x, int *__restrict__ region) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)kLists * (W + 1);
         t += (long long)gridDim.x * blockDim.x) {
        const int L = (int)(t / (W + 1)), g = (int)(t % (W + 1));
        region[t] = x[(long long)L * W + g];
    }
}

__global__ void k_in_bins(int n, const int *__restrict__ in_ptr, int cut1, int cut2, int *__restrict__ in_bin_of) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int deg = in_ptr[i + 1] - in_ptr[i];
        in_bin_of[i] = deg <= cut1 ? 0 : (deg <= cut2 ? 1 : 2);
    }
}

__global__ void k_iota(int n, int *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (int)i;
}

// number of pull chunk tasks of each long row
// ----------------------------------------------------------- generic scan

constexpr int kScanItems = 16;
constexpr int kScanBlock = 256 * kScanItems;

__global__ void k_scan_reduce(const int *__restrict__ in, long long m, int *__restrict__ sums) {
    long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < m) s += in[base + k];
    int total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single CTA: exclusive scan of the block sums, in place
__global__ void k_scan_top(int nb, int *__restrict__ sums) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        int total;
        int ex = block_excl_scan(v, &total);
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void k_scan_down(const int *__restrict__ in, long long m, const int *__restrict__ sums, int *__restrict__ out) {
    long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < m ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_excl_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < m) {
            out[base + k] = run;
            run += v[k];
        }
}

// out[0..m) = exclusive scan of in[0..m); out may alias in
di_status exclusive_scan(const int *in, int *out, long long m, cudaStream_t s) {
    if (m <= 0) return DI_OK;
    int nb = ceil_div(m, kScanBlock);
    int *sums = nullptr;
    DI_CUDA(cudaMallocAsync(&sums, sizeof(int) * (size_t)nb, s));
    k_scan_reduce<<<nb, 256, 0, s>>>(in, m, sums);
    k_scan_top<<<1, 256, 0, s>>>(nb, sums);
    k_scan_down<<<nb, 256, 0, s>>>(in, m, sums, out);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(sums, s);
    if (e != cudaSuccess) return cuda_fail(e, "exclusive_scan");
    return DI_OK;
}

// ------------------------------------------------- stable LSD radix pass

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;                       // per thread
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const int *__restrict__ keys, long long m, int shift,
                                                              int mask, int nb, int *__restrict__ hist, int ntiles) {
    __shared__ int h[257];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kRadixTile;
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        long long idx = base + it * kRadixThreads + threadIdx.x;
        if (idx < m) atomicAdd(&h[(keys[idx] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[(long long)b * ntiles + blockIdx.x] = h[b];
}

// Stable scatter: items of a tile keep their input order within each digit.
// Warp w owns items [tile + w*256, tile + (w+1)*256) in iterations of 32.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const int *__restrict__ keys_in,
                                                                 const int *__restrict__ vals_in,
                                                                 int *__restrict__ keys_out, int *__restrict__ vals_out,
                                                                 long long m, int shift, int mask, int nb,
                                                                 const int *__restrict__ offs, int ntiles) {
    __shared__ int wc[kRadixWarps][257];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = threadIdx.x; b < kRadixWarps * 257; b += blockDim.x) (&wc[0][0])[b] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kRadixTile + (long long)w * (32 * kRadixItems);
    int key[kRadixItems], val[kRadixItems], dig[kRadixItems], rnk[kRadixItems];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        long long idx = base + it * 32 + lane;
        bool ok = idx < m;
        key[it] = ok ? keys_in[idx] : 0;
        val[it] = ok ? vals_in[idx] : 0;
        dig[it] = ok ? ((key[it] >> shift) & mask) : nb;  // bucket nb collects the padding
        unsigned peers = __match_any_sync(kFull, dig[it]);
        int before = wc[w][dig[it]];
        __syncwarp();
        int r = __popc(peers & lt);
        if (r == 0) wc[w][dig[it]] = before + __popc(peers);
        __syncwarp();
        rnk[it] = before + r;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int run = 0;
        for (int ww = 0; ww < kRadixWarps; ++ww) {
            int t = wc[ww][b];
            wc[ww][b] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        if (dig[it] == nb) continue;
        long long pos = (long long)offs[(long long)dig[it] * ntiles + blockIdx.x] + wc[w][dig[it]] + rnk[it];
        keys_out[pos] = key[it];
        vals_out[pos] = val[it];
    }
}

// One stable counting-sort pass by digit (key >> shift) & mask, nb = mask + 1 <= 256 buckets.
di_status radix_pass(const int *keys_in, const int *vals_in, int *keys_out, int *vals_out, long long m, int shift,
                     int mask, cudaStream_t s) {
    if (m <= 0) return DI_OK;
    int nb = mask + 1;
    int ntiles = ceil_div(m, kRadixTile);
    long long hn = (long long)nb * ntiles;
    int *hist = nullptr;
    DI_CUDA(cudaMallocAsync(&hist, sizeof(int) * (size_t)hn, s));
    k_radix_hist<<<ntiles, kRadixThreads, 0, s>>>(keys_in, m, shift, mask, nb, hist, ntiles);
    di_status r = exclusive_scan(hist, hist, hn, s);
    if (r == DI_OK) {
        k_radix_scatter<<<ntiles, kRadixThreads, 0, s>>>(keys_in, vals_in, keys_out, vals_out, m, shift, mask, nb, hist,
                                                         ntiles);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(hist, s);
    if (r != DI_OK) return r;
    if (e != cudaSuccess) return cuda_fail(e, "radix_pass");
    return DI_OK;
}

// --------------------------------------------------------------- transpose

// source node of every edge position: the row whose range holds e.  A warp takes a tile of
// kExpandRuns x 32 consecutive positions, lane j the positions j, j + 32, ...: a binary search
// over all rows finds the row of its first one, and each later one is found by galloping
// forward from the previous row (a few loads, wherever empty rows lie between).
constexpr int kExpandRuns = 16;

__device__ __forceinline__ int row_from(const int *__restrict__ row_ptr, int n, long long e, int lo) {
    // row_ptr[lo] <= e < row_ptr[n]: the last r >= lo with row_ptr[r] <= e
    int hi = lo + 1;
    long long step = 1;
    while (hi < n && (long long)row_ptr[hi] <= e) {
        lo = hi;
        step <<= 1;
        hi = (int)min((long long)n, (long long)lo + step);
    }
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if ((long long)row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_expand_rows(int n, long long nnz, const int *__restrict__ row_ptr, int *__restrict__ src) {
    const int lane = threadIdx.x & 31;
    const long long tile = 32LL * kExpandRuns, tiles = (nnz + tile - 1) / tile;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles; t += nw) {
        int r = 0;
        for (int k = 0; k < kExpandRuns; ++k) {
            const long long e = t * tile + 32LL * k + lane;
            if (e >= nnz) break;
            r = row_from(row_ptr, n, e, r);  // rows only move forward along the lane's positions
            src[e] = r;
        }
    }
}

// In-degrees.  On power-law graphs a few targets take percents of all edges and their
// global atomics serialize in one L2 slice, so each CTA first counts its tile of kCountTile
// edges in a small shared-memory hash table (open addressing, a few probes) and adds each
// table entry to global memory once; targets that find no slot go straight to global memory.
// A column outside [0, n) is not counted; it sets kColRange in *flags (when flags is given).
constexpr int kCountTile = 4096, kCountSlots = 2048, kCountProbes = 4;

__global__ void __launch_bounds__(256) k_count_in(long long nnz, const int *__restrict__ col_idx, int n,
                                                  int *__restrict__ indeg, int *__restrict__ flags) {
    __shared__ int s_key[kCountSlots], s_cnt[kCountSlots];
    bool bad = false;
    for (long long t0 = (long long)blockIdx.x * kCountTile; t0 < nnz; t0 += (long long)gridDim.x * kCountTile) {
        for (int k = threadIdx.x; k < kCountSlots; k += blockDim.x) {
            s_key[k] = -1;
            s_cnt[k] = 0;
        }
        __syncthreads();
        const long long t1 = min(nnz, t0 + kCountTile);
        for (long long e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
            const int j = col_idx[e];
            if ((unsigned)j >= (unsigned)n) {
                bad = true;
                continue;
            }
            unsigned h = ((unsigned)j * 2654435761u) >> 21;  // 11 bits: kCountSlots = 2048
            bool done = false;
            for (int p = 0; p < kCountProbes && !done; ++p) {
                const int slot = (h + p) & (kCountSlots - 1);
                const int prev = atomicCAS(&s_key[slot], -1, j);
                if (prev == -1 || prev == j) {
                    atomicAdd(&s_cnt[slot], 1);
                    done = true;
                }
            }
            if (!done) atomicAdd(&indeg[j], 1);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kCountSlots; k += blockDim.x)
            if (s_key[k] >= 0) atomicAdd(&indeg[s_key[k]], s_cnt[k]);
        __syncthreads();
    }
    if (bad && flags) atomicOr(flags, kColRange);
}


// ---- the hot targets: the k largest in-degrees, ties by lower id, without sorting all n
//
// A most-significant-digit-first radix select finds t, the k-th largest in-degree: four
// passes over the in-degrees, each a 256-bin histogram of one byte among the nodes whose
// higher bytes match the prefix found so far, and a one-thread step that picks the bin
// holding the k-th largest.  The nodes above t (fewer than k) and the first k - #above
// nodes equal to t in id order (an ordered compaction) are then sorted by (in-degree
// descending, id ascending) in one CTA.

struct HotSel {
    unsigned prefix;  // the bytes of t found so far (high bits)
    int need;         // how many of the k still lie at or below the current prefix
    int above;        // nodes with in-degree > t (after the last pass)
    int ncand;        // candidates written
};

__global__ void k_hot_hist(int n, const int *__restrict__ indeg, int pass, const HotSel *__restrict__ hs,
                           unsigned *__restrict__ hist) {
    __shared__ unsigned h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const int shift = 24 - 8 * pass;
    const unsigned pre = hs->prefix;
    const unsigned hmask = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned v = (unsigned)indeg[i];
        if ((v & hmask) == pre) atomicAdd(&h[(v >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// one thread: the bin of this pass that holds the need-th largest; clears the histogram
__global__ void k_hot_pick(int pass, HotSel *__restrict__ hs, unsigned *__restrict__ hist) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int shift = 24 - 8 * pass;
    int need = hs->need;
    int b = 255;
    for (; b > 0; --b) {
        const int c = (int)hist[b];
        if (c >= need) break;
        need -= c;
    }
    hs->prefix |= (unsigned)b << shift;
    hs->need = need;  // the need-th largest among the nodes of bin b
    for (int j = 0; j < 256; ++j) hist[j] = 0u;
}

constexpr int kTieBlock = 4096;  // ids per block of the ordered tie compaction

// nodes above t go to the candidates (any order); per block of ids, the number equal to t
__global__ void k_hot_above(int n, const int *__restrict__ indeg, HotSel *__restrict__ hs, int *__restrict__ cand,
                            int cap, int *__restrict__ ties) {
    __shared__ int s_t;
    if (threadIdx.x == 0) s_t = 0;
    __syncthreads();
    const int t = (int)hs->prefix;
    const long long beg = (long long)blockIdx.x * kTieBlock, end = min((long long)n, beg + kTieBlock);
    int c = 0;
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const int v = indeg[i];
        if (v > t) {
            const int at = atomicAdd(&hs->above, 1);
            if (at < cap) cand[at] = (int)i;
        } else if (v == t) {
            ++c;
        }
    }
    if (c) atomicAdd(&s_t, c);
    __syncthreads();
    if (threadIdx.x == 0) ties[blockIdx.x] = s_t;
}

// the first (k - above) nodes equal to t, in id order, after the nodes above t
__global__ void k_hot_ties(int n, int k, const int *__restrict__ indeg, const HotSel *__restrict__ hs,
                           const int *__restrict__ tie_off, int *__restrict__ cand) {
    __shared__ int s_w[32];
    const int t = (int)hs->prefix, above = min(hs->above, k), want = k - above;
    int base = tie_off[blockIdx.x];
    if (base >= want) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long beg = (long long)blockIdx.x * kTieBlock, end = min((long long)n, beg + kTieBlock);
    for (long long i0 = beg; i0 < end && base < want; i0 += blockDim.x) {
        const long long i = i0 + threadIdx.x;
        const bool is = i < end && indeg[i] == t;
        const unsigned bal = __ballot_sync(0xffffffffu, is);
        if (lane == 0) s_w[w] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int j = 0; j < nw; ++j) {
            off += j < w ? s_w[j] : 0;
            tot += s_w[j];
        }
        const int r = base + off + __popc(bal & ((1u << lane) - 1u));
        if (is && r < want) cand[above + r] = (int)i;
        base += tot;
        __syncthreads();
    }
}

// one CTA of kHotSlots threads: sort the k candidates by (in-degree descending, id ascending)
// and count those with at least min_deg in-links
__global__ void k_hot_sort(int k, const int *__restrict__ indeg, const int *__restrict__ cand, int min_deg,
                           int *__restrict__ hot_ids, int *__restrict__ count) {
    __shared__ long long key[kHotSlots];
    const int t = threadIdx.x;
    // larger in-degree first, then lower id: sort ascending on (-indeg, id)
    key[t] = t < k ? ((long long)(0x7fffffff - indeg[cand[t]]) << 32) | (unsigned)cand[t] : LLONG_MAX;
    __syncthreads();
    for (int size = 2; size <= kHotSlots; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int j = t ^ stride;
            if (j > t) {
                const bool up = (t & size) == 0;
                const long long a = key[t], b = key[j];
                if ((a > b) == up) {
                    key[t] = b;
                    key[j] = a;
                }
            }
            __syncthreads();
        }
    }
    int c = 0;
    if (t < k) {
        const int id = (int)(key[t] & 0xffffffffLL);
        hot_ids[t] = id;
        c = indeg[id] >= min_deg ? 1 : 0;
    }
    const int total = __syncthreads_count(c);
    if (t == 0) *count = total;  // the qualifying ones are a prefix of the sorted order
}


// flag[i] = 1 everywhere, then 0 for the first k ids of the in-degree order (the hot targets)
__global__ void k_hot_flags(int n, int *__restrict__ flag) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        flag[i] = 1;
}

__global__ void k_mark_hot(int k, const int *__restrict__ by_indeg, int *__restrict__ flag) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) flag[by_indeg[r]] = 0;
}

__global__ void k_inverse(int n, const int *__restrict__ perm, int *__restrict__ inv) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        inv[perm[r]] = (int)r;
}

// out-degree of internal node r (the input node perm[r]); deg[n] = 0 so a scan gives row_ptr
__global__ void k_perm_deg(int n, const int *__restrict__ perm, const int *__restrict__ row_ptr, int *__restrict__ deg) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += (long long)gridDim.x * blockDim.x)
        deg[r] = r < n ? row_ptr[perm[r] + 1] - row_ptr[perm[r]] : 0;
}

// The internal numbering puts the nh <= kHotSlots hot targets first and keeps every other
// node in input order, so the relabeled CSR is the input CSR with nh rows moved to the front.
// Its edges come from nh + 1 runs of the input: the hot rows, then the input with those rows
// cut out -- nh + 1 segments between them.  k_hot_segments builds that table (one CTA):
//   tab[0 .. nh]            hot row k's first input edge (k < nh)
//   tab[kSeg .. kSeg+nh]    non-hot segment k's first input edge
//   tab[2kSeg .. 2kSeg+nh+1] edges of the non-hot segments before segment k (a prefix)
constexpr int kSeg = kHotSlots + 2;

__global__ void __launch_bounds__(kHotSlots) k_hot_segments(int nh, long long nnz, const int *__restrict__ hot,
                                                           const int *__restrict__ row_ptr_in, int *__restrict__ tab) {
    __shared__ int s_sorted[kHotSlots];
    __shared__ int s_len[kHotSlots + 1];
    const int t = threadIdx.x;
    // hot ids in ascending input order: each id's rank among them (ids are distinct)
    if (t < nh) {
        const int h = hot[t];
        int rank = 0;
        for (int j = 0; j < nh; ++j) rank += hot[j] < h;
        s_sorted[rank] = h;
        tab[t] = row_ptr_in[h];
    }
    __syncthreads();
    // non-hot segment k: from the end of the (k-1)-th hot row (input order) to the start of the k-th
    for (int k = t; k <= nh; k += blockDim.x) {
        const int a = k == 0 ? 0 : row_ptr_in[s_sorted[k - 1] + 1];
        const int b = k == nh ? (int)nnz : row_ptr_in[s_sorted[k]];
        tab[kSeg + k] = a;
        s_len[k] = b - a;
    }
    __syncthreads();
    if (t == 0) {
        int c = 0;
        for (int k = 0; k <= nh; ++k) {
            tab[2 * kSeg + k] = c;
            c += s_len[k];
        }
        tab[2 * kSeg + nh + 1] = c;
    }
}

// edge e of the relabeled CSR copies one input edge, its column renumbered: in a hot row k
// (e below the hot rows' total) edge e - row_ptr_out[k] of that row, else the (e - hot total)-th
// edge of the input outside the hot rows, found in the segment table (shared memory)
__global__ void __launch_bounds__(256) k_perm_cols(int nh, long long nnz, const int *__restrict__ tab,
                                                   const int *__restrict__ new_of, const int *__restrict__ col_in,
                                                   const int *__restrict__ row_ptr_out, int *__restrict__ col_out) {
    __shared__ int s_hot_out[kHotSlots + 1], s_hot_in[kHotSlots], s_seg[kHotSlots + 1], s_cum[kHotSlots + 2];
    for (int k = threadIdx.x; k <= nh + 1; k += blockDim.x) {
        if (k <= nh) s_hot_out[k] = row_ptr_out[k];
        if (k < nh) s_hot_in[k] = tab[k];
        if (k <= nh) s_seg[k] = tab[kSeg + k];
        s_cum[k] = tab[2 * kSeg + k];
    }
    __syncthreads();
    const long long hot_total = s_hot_out[nh];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x) {
        long long src_e;
        if (e < hot_total) {
            int lo = 0, hi = nh;  // the last hot row k < nh with row_ptr_out[k] <= e
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_hot_out[mid] <= e) lo = mid; else hi = mid;
            }
            src_e = (long long)s_hot_in[lo] + (e - s_hot_out[lo]);
        } else {
            const long long o = e - hot_total;
            int lo = 0, hi = nh + 1;  // the last segment k <= nh with cum[k] <= o (it is not empty)
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_cum[mid] <= o) lo = mid; else hi = mid;
            }
            src_e = (long long)s_seg[lo] + (o - s_cum[lo]);
        }
        col_out[e] = new_of[col_in[src_e]];
    }
}

__global__ void k_perm_values(int n, const int *__restrict__ perm, const double *__restrict__ in, double *__restrict__ out) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        out[r] = in[perm[r]];
}

int grid_for(long long work, int threads, int num_sms) {
    long long b = (work + threads - 1) / threads;
    long long cap = (long long)num_sms * 16;
    return (int)std::max(1LL, std::min(b, cap));
}

}  // namespace

di_status validate_v(di_graph *g, const double *V_dev) {
    cudaStream_t s = g->stream;
    struct Tmp { int flags; int pad; double sum; };
    Tmp *t = nullptr;
    DI_CUDA(cudaMallocAsync(&t, sizeof(Tmp), s));
    DI_CUDA(cudaMemsetAsync(t, 0, sizeof(Tmp), s));
    k_validate_v<<<grid_for(g->n, 256, g->num_sms), 256, 0, s>>>(g->n, V_dev, &t->flags, &t->sum);
    Tmp h{};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, t, sizeof(Tmp), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(t, s);
    if (e != cudaSuccess) return cuda_fail(e, "validate V");
    if (h.flags & kVNonFinite) return set_error(DI_EINVAL, "V has a NaN or infinite entry");
    if (h.flags & kVNeg) return set_error(DI_EINVAL, "V has a negative entry");
    if (!(fabs(h.sum - 1.0) <= 1e-12))
        return set_error(DI_EINVAL, "V must be normalized: |V|_1 = " + std::to_string(h.sum));
    return DI_OK;
}

// 64-bit fingerprint of every input row (its out-degree and its targets in order), kept in
// input numbering: a graph update compares the fingerprints of two graphs to find the rows
// whose out-links changed (Section 3.2: only those rows inject fluid).  SplitMix64 mixing.
__device__ __forceinline__ unsigned long long fp_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// fingerprint = mix(#out, sum over the row's positions p of mix(target_p, p)): the sum lets a
// warp share a long row; the position term keeps it order-sensitive
__device__ __forceinline__ unsigned long long fp_edge(int t, int p) {
    return fp_mix(((unsigned long long)(unsigned)t << 32 | (unsigned)p) + 0x9e3779b97f4a7c15ull);
}

// the fingerprint of every input row, from the relabeled CSR: internal row r is input row
// perm[r] with its targets renumbered and their order kept, so perm maps both back
__global__ void k_row_hash(int n, const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                           const int *__restrict__ perm, unsigned long long *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int w0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; w0 < n; w0 += nw * 32) {
        const int v = w0 + lane;
        int beg = 0, deg = 0;
        unsigned long long acc = 0;
        if (v < n) {
            beg = row_ptr[v];
            deg = row_ptr[v + 1] - beg;
            if (deg <= 64)
                for (int p = 0; p < deg; ++p) acc += fp_edge(perm[col_idx[beg + p]], p);
        }
        // rows above 64 out-links: the whole warp, one row at a time
        unsigned longs = __ballot_sync(0xffffffffu, v < n && deg > 64);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int b = __shfl_sync(0xffffffffu, beg, src), dg = __shfl_sync(0xffffffffu, deg, src);
            unsigned long long part = 0;
            for (int p = lane; p < dg; p += 32) part += fp_edge(perm[col_idx[b + p]], p);
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == src) acc = part;
        }
        if (v < n) out[perm[v]] = fp_mix(0x243f6a8885a308d3ull ^ (unsigned long long)deg) + acc;
    }
}

int count_grid(const di_graph *g, long long L) {
    return (int)std::max(1LL, std::min((L + kCountTile - 1) / kCountTile, (long long)g->num_sms * 8));
}

constexpr int kCopyChunks = 8;  // pieces of a host col_idx, each counted as soon as it lands

// in-degrees of g->col_idx into indeg (zeroed), column range errors into *flags.  From a host
// col_idx the copy runs on the second stream in kCopyChunks pieces; the first stream counts each
// piece after its copy, so the counting of one piece overlaps the copy of the next.
cudaError_t count_columns(di_graph *g, const int *col_host, int *indeg, int *flags) {
    cudaStream_t s = g->stream;
    const long long L = g->nnz;
    if (!col_host) {
        k_count_in<<<count_grid(g, L), 256, 0, s>>>(L, g->col_idx, g->n, indeg, flags);
        return cudaGetLastError();
    }
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    // the copies start after the first stream's work so far (the allocation of col_idx)
    e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cap, ev, 0);
    const long long step = ceil_div(ceil_div(L, (long long)kCopyChunks), (long long)kCountTile) * kCountTile;
    for (long long a = 0; e == cudaSuccess && a < L; a += step) {
        const long long m = std::min(step, L - a);
        e = cudaMemcpyAsync(g->col_idx + a, col_host + a, sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, g->cap);
        if (e == cudaSuccess) e = cudaEventRecord(ev, g->cap);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        if (e == cudaSuccess) {
            k_count_in<<<count_grid(g, m), 256, 0, s>>>(m, g->col_idx + a, g->n, indeg, flags);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) cudaStreamSynchronize(g->cap);  // no copy may still be writing after a failure
    cudaEventDestroy(ev);
    return e;
}

di_status build_graph(di_graph *g, const int *col_host) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    const long long L = g->nnz;

    // 1. validation and in-degrees: k_validate_rows checks the row starts, the in-degree count
    //    the columns (it reads each of them once); one host check of the flags after both
    int *indeg = nullptr;
    {
        int *flags = nullptr;
        DI_CUDA(cudaMallocAsync(&flags, sizeof(int), s));
        DI_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
        DI_CUDA(cudaMallocAsync(&indeg, sizeof(int) * (size_t)n, s));
        DI_CUDA(cudaMemsetAsync(indeg, 0, sizeof(int) * (size_t)n, s));
        k_validate_rows<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, L, g->row_ptr, flags);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && L > 0) e = count_columns(g, col_host, indeg, flags);
        int hf = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(flags, s);
        if (e == cudaSuccess && hf) cudaFreeAsync(indeg, s);
        if (e != cudaSuccess) return cuda_fail(e, "validate CSR");
        if (hf & kBadRowPtr0) return set_error(DI_EINVAL, "row_ptr[0] must be 0");
        if (hf & kBadRowPtrN) return set_error(DI_EINVAL, "row_ptr[n] must equal nnz");
        if (hf & kNotMonotone) return set_error(DI_EINVAL, "row_ptr must be non-decreasing");
        if (hf & kColRange) return set_error(DI_EINVAL, "col_idx has an entry outside [0, n)");
    }

    // 1b. internal numbering: the hot targets -- the kHotSlots largest in-degrees (at least
    //     kHotMinInDeg), ties by lower input id, found by a radix select -- become ids
    //     0..n_hot-1; every other node keeps its input order after them.  The push sums the
    //     hot targets' fluid in shared memory with a single compare; the rest stay spread over
    //     the L2 slices as the input spreads them.
    {
        int *ka = nullptr, *kb = nullptr, *va = nullptr, *vb = nullptr, *cnt = nullptr;
        DI_CUDA(cudaMallocAsync(&ka, sizeof(int) * (size_t)n, s));
        DI_CUDA(cudaMallocAsync(&kb, sizeof(int) * (size_t)n, s));
        DI_CUDA(cudaMallocAsync(&va, sizeof(int) * (size_t)n, s));
        DI_CUDA(cudaMallocAsync(&vb, sizeof(int) * (size_t)n, s));
        DI_CUDA(cudaMallocAsync(&cnt, sizeof(int), s));
        // the k largest in-degrees (ties by lower id): radix select, then one small sort
        const int k = std::min(kHotSlots, n);
        DI_CUDA(cudaMallocAsync(&g->hot_ids, sizeof(int) * kHotSlots, s));
        {
            HotSel *hs = nullptr;
            unsigned *hist = nullptr;
            int *cand = nullptr, *ties = nullptr;
            const int nblk = ceil_div(n, kTieBlock);
            DI_CUDA(cudaMallocAsync(&hs, sizeof(HotSel), s));
            DI_CUDA(cudaMallocAsync(&hist, sizeof(unsigned) * 256, s));
            DI_CUDA(cudaMallocAsync(&cand, sizeof(int) * kHotSlots, s));
            DI_CUDA(cudaMallocAsync(&ties, sizeof(int) * (size_t)(nblk + 1), s));
            HotSel h0 = {0u, k, 0, 0};
            DI_CUDA(cudaMemcpyAsync(hs, &h0, sizeof(HotSel), cudaMemcpyHostToDevice, s));
            DI_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned) * 256, s));
            for (int pass = 0; pass < 4; ++pass) {
                k_hot_hist<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, indeg, pass, hs, hist);
                k_hot_pick<<<1, 32, 0, s>>>(pass, hs, hist);
            }
            k_hot_above<<<nblk, 256, 0, s>>>(n, indeg, hs, cand, kHotSlots, ties);
            di_status r = exclusive_scan(ties, ties, nblk, s);
            if (r != DI_OK) return r;
            k_hot_ties<<<nblk, 256, 0, s>>>(n, k, indeg, hs, ties, cand);
            k_hot_sort<<<1, kHotSlots, 0, s>>>(k, indeg, cand, kHotMinInDeg, g->hot_ids, cnt);
            cudaFreeAsync(hs, s);
            cudaFreeAsync(hist, s);
            cudaFreeAsync(cand, s);
            cudaFreeAsync(ties, s);
        }
        int hk = 0;
        DI_CUDA(cudaMemcpyAsync(&hk, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        g->n_hot = hk;
        // perm: the hot ids in in-degree order, then every other id ascending (a stable
        // two-bucket pass on "not hot" puts the hot ids first; they are then overwritten
        // with their in-degree order)
        k_hot_flags<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, kb);           // kb[i] = 1
        if (hk > 0) k_mark_hot<<<1, 256, 0, s>>>(hk, g->hot_ids, kb);              // kb[hot] = 0
        k_iota<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, vb);
        {
            di_status r = radix_pass(kb, vb, ka, va + 0, n, 0, 1, s);  // va <- ids, hot first (ascending)
            if (r != DI_OK) return r;
        }
        if (hk > 0) DI_CUDA(cudaMemcpyAsync(va, g->hot_ids, sizeof(int) * hk, cudaMemcpyDeviceToDevice, s));
        g->perm = va;
        DI_CUDA(cudaMallocAsync(&g->new_of, sizeof(int) * (size_t)n, s));
        k_inverse<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, g->perm, g->new_of);
        // relabeled CSR
        int *rp2 = nullptr, *ci2 = nullptr;
        DI_CUDA(cudaMallocAsync(&rp2, sizeof(int) * (size_t)(n + 1), s));
        // kColPad ints past the last link: the push stages hub rows with 16-byte bulk copies
        // whose end is rounded up
        DI_CUDA(cudaMallocAsync(&ci2, sizeof(int) * (size_t)(std::max<long long>(L, 1) + kColPad), s));
        DI_CUDA(cudaMemsetAsync(ci2 + std::max<long long>(L, 1), 0, sizeof(int) * kColPad, s));
        k_perm_deg<<<grid_for((long long)n + 1, 256, g->num_sms), 256, 0, s>>>(n, g->perm, g->row_ptr, rp2);
        di_status r = exclusive_scan(rp2, rp2, (long long)n + 1, s);
        if (r != DI_OK) return r;
        if (L > 0) {
            int *tab = nullptr;
            DI_CUDA(cudaMallocAsync(&tab, sizeof(int) * 3 * kSeg, s));
            k_hot_segments<<<1, kHotSlots, 0, s>>>(hk, L, g->hot_ids, g->row_ptr, tab);
            k_perm_cols<<<grid_for(L, 256, g->num_sms), 256, 0, s>>>(hk, L, tab, g->new_of, g->col_idx, rp2, ci2);
            cudaFreeAsync(tab, s);
        }
        cudaFreeAsync(g->row_ptr, s);
        cudaFreeAsync(g->col_idx, s);
        g->row_ptr = rp2;
        g->col_idx = ci2;
        if (g->V) {
            double *v2 = nullptr;
            DI_CUDA(cudaMallocAsync(&v2, sizeof(double) * (size_t)n, s));
            k_perm_values<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, g->perm, g->V, v2);
            cudaFreeAsync(g->V, s);
            g->V = v2;
        }
        cudaFreeAsync(indeg, s);
        cudaFreeAsync(ka, s);
        cudaFreeAsync(kb, s);
        cudaFreeAsync(vb, s);
        cudaFreeAsync(cnt, s);
        DI_CUDA(cudaGetLastError());
    }

    // 2. out-degree classes and the per-warp frontier regions of the sweep scan
    // one wave of scan CTAs (every chunk resident at once), at most kMaxScanBlocks
    g->G = std::max(1, std::min(std::min(kMaxScanBlocks, g->num_sms * scan_blocks_per_sm()), ceil_div(n, kChunkAlign)));
    g->chunk = ceil_div(ceil_div(n, g->G), kChunkAlign) * kChunkAlign;
    g->G = ceil_div(n, g->chunk);
    g->W = g->G * kWarps;
    const long long npad = (long long)g->G * g->chunk;
    DI_CUDA(cudaMallocAsync(&g->bin_of, sizeof(int) * (size_t)n, s));
    DI_CUDA(cudaMallocAsync(&g->cls, (size_t)npad, s));
    DI_CUDA(cudaMemsetAsync(g->cls, 0, (size_t)npad, s));
    DI_CUDA(cudaMallocAsync(&g->inv_deg, sizeof(double) * (size_t)n, s));
    DI_CUDA(cudaMallocAsync(&g->inv_deg32, sizeof(float) * (size_t)n, s));
    DI_CUDA(cudaMallocAsync(&g->rec64, sizeof(RowRec<double>) * (size_t)n, s));
    DI_CUDA(cudaMallocAsync(&g->rec32, sizeof(RowRec<float>) * (size_t)n, s));
    {
        const int W = g->W;
        DI_CUDA(cudaMallocAsync(&g->region, sizeof(int) * kLists * (size_t)(W + 1), s));
        DI_CUDA(cudaMallocAsync(&g->fcount, sizeof(int) * kCountRows * (size_t)W, s));
        DI_CUDA(cudaMemsetAsync(g->fcount, 0, sizeof(int) * kCountRows * (size_t)W, s));
        DI_CUDA(cudaMallocAsync(&g->pre, sizeof(int) * kCountRows * (size_t)(W + 1), s));
        DI_CUDA(cudaMemsetAsync(g->pre, 0, sizeof(int) * kCountRows * (size_t)(W + 1), s));
    }
    {
        di_status r = set_out_classes(g, kOutCut1, kOutCut2);
        if (r != DI_OK) return r;
    }

    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

// Out-degree classes (0 dangling, 1 up to cut1 out-links, 2 up to cut2, 3 above; the class byte
// of a class-3 node is 2 + the number of chunks its row is pushed in), the packed
// row records, and the per-warp frontier regions of the sweep scan for those classes.  Run at
// creation and again when the autotuner changes the cutoffs; the buffers keep their sizes (the
// regions of all classes together always hold n entries), so captured loops stay valid.
di_status set_out_classes(di_graph *g, int cut1, int cut2) {
    cudaStream_t s = g->stream;
    const int n = g->n;
    g->cut1 = cut1;
    g->cut2 = cut2;
    double *tab = nullptr;
    DI_CUDA(cudaMallocAsync(&tab, sizeof(double) * kInvTable, s));
    k_inv_table<<<kInvTable / 256, 256, 0, s>>>(g->d, tab);
    k_out_bins<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(n, g->row_ptr, cut1, cut2, g->d, tab, g->bin_of, g->cls,
                                                           g->inv_deg, g->inv_deg32, g->rec64, g->rec32);
    cudaFreeAsync(tab, s);
    const int W = g->W;
    int *cnt = nullptr;
    DI_CUDA(cudaMallocAsync(&cnt, sizeof(int) * (kLists * (size_t)W + 1), s));
    DI_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (kLists * (size_t)W + 1), s));
    k_sub_counts<<<W, 256, 0, s>>>(n, g->chunk / kWarps, g->cls, cnt, W);
    {
        di_status r = exclusive_scan(cnt, cnt, (long long)kLists * W + 1, s);
        if (r != DI_OK) return r;
    }
    k_region_layout<<<grid_for((long long)kLists * (W + 1), 256, g->num_sms), 256, 0, s>>>(W, cnt, g->region);
    std::vector<int> h(kLists * (size_t)(W + 1));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), g->region, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(cnt, s);
    if (e != cudaSuccess) return cuda_fail(e, "frontier regions");
    long long prev = 0;
    for (int L = 0; L < kLists; ++L) {
        long long end = h[(size_t)L * (W + 1) + W];
        g->bin_count[L] = (int)(end - prev);
        prev = end;
    }
    return DI_OK;
}

// The in-link side (power iteration, exports, ALGO-OP weights), built at its first use:
// a solve never reads it.
di_status build_transpose(di_graph *g) {
    if (g->transposed) return DI_OK;
    cudaStream_t s = g->stream;
    // what an earlier attempt that failed part-way left behind
    void *partial[] = {g->in_ptr, g->in_src};
    for (void *b : partial)
        if (b) cudaFreeAsync(b, s);
    g->in_ptr = g->in_src = nullptr;
    const int n = g->n;
    const long long L = g->nnz;
    // 3. in-link CSR: stable LSD radix sort of (target, source) pairs in source order
    DI_CUDA(cudaMallocAsync(&g->in_ptr, sizeof(int) * (size_t)(n + 1), s));
    DI_CUDA(cudaMallocAsync(&g->in_src, sizeof(int) * (size_t)std::max<long long>(L, 1), s));
    DI_CUDA(cudaMemsetAsync(g->in_ptr, 0, sizeof(int) * (size_t)(n + 1), s));
    if (L > 0) {
        k_count_in<<<count_grid(g, L), 256, 0, s>>>(L, g->col_idx, n, g->in_ptr, nullptr);
        int *ka = nullptr, *kb = nullptr, *va = nullptr, *vtmp = nullptr;
        DI_CUDA(cudaMallocAsync(&ka, sizeof(int) * (size_t)L, s));
        DI_CUDA(cudaMallocAsync(&kb, sizeof(int) * (size_t)L, s));
        DI_CUDA(cudaMallocAsync(&va, sizeof(int) * (size_t)L, s));
        DI_CUDA(cudaMallocAsync(&vtmp, sizeof(int) * (size_t)L, s));
        DI_CUDA(cudaMemcpyAsync(ka, g->col_idx, sizeof(int) * (size_t)L, cudaMemcpyDeviceToDevice, s));
        k_expand_rows<<<grid_for(L, 256, g->num_sms), 256, 0, s>>>(n, L, g->row_ptr, va);
        int bits = 1;
        while (bits < 31 && (1LL << bits) < (long long)n) ++bits;
        int passes = (bits + 7) / 8;
        // keys ping-pong between ka and kb; values alternate between va and vtmp and
        // the last pass writes them into in_src
        int *kin = ka, *kout = kb, *vin = va, *vout = nullptr;
        for (int p = 0; p < passes; ++p) {
            bool last = (p == passes - 1);
            vout = last ? g->in_src : (vin == va ? vtmp : va);
            di_status r = radix_pass(kin, vin, kout, vout, L, 8 * p, 0xff, s);
            if (r != DI_OK) return r;
            std::swap(kin, kout);
            vin = vout;
        }
        cudaFreeAsync(ka, s);
        cudaFreeAsync(kb, s);
        cudaFreeAsync(va, s);
        cudaFreeAsync(vtmp, s);
    }
    {
        di_status r = exclusive_scan(g->in_ptr, g->in_ptr, (long long)n + 1, s);
        if (r != DI_OK) return r;
    }

    DI_CUDA(cudaGetLastError());
    g->transposed = true;
    return DI_OK;
}

// row fingerprints, at the first graph update that reads them
di_status ensure_rowhash(di_graph *g) {
    if (g->rowhash) return DI_OK;
    DI_CUDA(cudaMallocAsync(&g->rowhash, sizeof(unsigned long long) * (size_t)g->n, g->stream));
    k_row_hash<<<std::max(1, std::min(ceil_div(g->n, 256), g->num_sms * 8)), 256, 0, g->stream>>>(
        g->n, g->row_ptr, g->col_idx, g->perm, g->rowhash);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

// in-degree class of every node (0 up to kInCut1 in-links, 1 up to kInCut2, 2 above) into a
// device buffer of n ints; the in-link CSR must exist
di_status in_degree_classes(di_graph *g, int *out_dev) {
    k_in_bins<<<grid_for(g->n, 256, g->num_sms), 256, 0, g->stream>>>(g->n, g->in_ptr, kInCut1, kInCut2, out_dev);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

di_status build_in_dst(di_graph *g) {
    if (g->in_dst) return DI_OK;
    di_status r = build_transpose(g);
    if (r != DI_OK) return r;
    const long long L = g->nnz;
    DI_CUDA(cudaMallocAsync(&g->in_dst, sizeof(int) * (size_t)std::max<long long>(L, 1), g->stream));
    if (L > 0) k_expand_rows<<<grid_for(L, 256, g->num_sms), 256, 0, g->stream>>>(g->n, L, g->in_ptr, g->in_dst);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

}  // namespace diter
