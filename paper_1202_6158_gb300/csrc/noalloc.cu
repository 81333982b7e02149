// noalloc.cu -- a power iteration that allocates no device memory.
//
// Some callers cannot call cudaMalloc at all: services that must not grow their
// device memory after start-up or that hand out device memory only from their
// own pre-sized pools, and plug-ins loaded into a host program that owns the
// GPU's allocator.  di_power_noalloc serves them: it computes the same power
// iteration as di_power (X_0 = 0, X_{k+1} = dPX_k + (1-d)/n, stop when
// |X_{k+1} - X_k|_1 * d/(1-d) < tol) directly on device arrays the caller
// already owns, and keeps its working memory -- the two buffers of d*x/outdeg,
// the per-CTA partial sums and a small control block -- in one fixed-size
// static __device__ array.  The array is committed on a GPU when this file's
// module is loaded there; with CUDA's lazy module loading that is the first
// call on that GPU, so a caller that must not grow its footprint later makes
// one call during its own start-up.  It then stays until the process exits.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace diter {
namespace {

constexpr int kNaMaxN = 1 << 16;        // largest graph (nodes) the static array holds
constexpr int kNaThreads = 256;
constexpr int kNaMaxParts = 256;        // CTAs of the pull kernel, at most
constexpr int kNaBatch = 16;            // products launched between two host checks

struct NaState {
    double delta;  // |X_{k+1} - X_k|_1 of the last product
    int iters;
    int done;      // 1 stop rule met, 2 limit reached, 3 non-finite
    int cur;       // which buffer holds d*x/outdeg of the current iterate
    int flags;     // input checks: 1 bad in_ptr, 2 bad row_ptr, 4 source id out of range
};

// layout: control block, partials, then two n-sized buffers
constexpr size_t kNaOffParts = 256;
constexpr size_t kNaOffZ0 = kNaOffParts + sizeof(double) * kNaMaxParts;
constexpr size_t kNaOffZ1 = kNaOffZ0 + sizeof(double) * kNaMaxN;
constexpr size_t kNaBytes = kNaOffZ1 + sizeof(double) * kNaMaxN;

// The scratch.  Every call shares it and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

// CSR checks in two steps: the row pointers first (they bound everything else)
__global__ void k_na_check_ptrs(int n, long long nnz, const int *__restrict__ in_ptr, const int *__restrict__ row_ptr,
                                NaState *st) {
    int f = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (in_ptr[0] != 0 || (long long)in_ptr[n] != nnz) f |= 1;
        if (row_ptr[0] != 0 || (long long)row_ptr[n] != nnz) f |= 2;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (in_ptr[i + 1] < in_ptr[i]) f |= 1;
        if (row_ptr[i + 1] < row_ptr[i]) f |= 2;
    }
    if (f) atomicOr(&st->flags, f);
}

__global__ void k_na_check_src(int n, long long nnz, const int *__restrict__ in_src, NaState *st) {
    int f = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
        if (in_src[k] < 0 || in_src[k] >= n) f |= 4;
    if (f) atomicOr(&st->flags, f);
}

__global__ void k_na_init(int n, double *__restrict__ X, double *__restrict__ Z0, double *__restrict__ Z1,
                          NaState *st) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        X[i] = 0.0;
        Z0[i] = 0.0;
        Z1[i] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->delta = 0.0;
        st->iters = 0;
        st->done = 0;
        st->cur = 0;
    }
}

// one product, a thread per row: y_j = (1-d)/n + sum_{i -> j} d*x_i/outdeg(i)
__global__ void __launch_bounds__(kNaThreads) k_na_pull(int n, const int *__restrict__ in_ptr,
                                                        const int *__restrict__ in_src,
                                                        const int *__restrict__ row_ptr, double d,
                                                        double *__restrict__ X, double *__restrict__ Z0,
                                                        double *__restrict__ Z1, double *__restrict__ parts,
                                                        const NaState *__restrict__ st) {
    __shared__ double sh[kNaThreads / 32];
    if (st->done) return;
    const double *zc = st->cur ? Z1 : Z0;
    double *zn = st->cur ? Z0 : Z1;
    const double base = (1.0 - d) / (double)n;
    double delta = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = in_ptr[j]; k < in_ptr[j + 1]; ++k) acc += zc[in_src[k]];
        const double y = base + acc;
        delta += fabs(y - X[j]);
        X[j] = y;
        const int deg = row_ptr[j + 1] - row_ptr[j];
        zn[j] = deg ? (d * y) / (double)deg : 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) delta += __shfl_down_sync(0xffffffffu, delta, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = delta;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) a += sh[k];
        parts[blockIdx.x] = a;
    }
}

__global__ void k_na_finalize(int nparts, const double *__restrict__ parts, double d, double tol, int max_iter,
                              NaState *st) {
    if (threadIdx.x != 0 || st->done) return;
    double a = 0.0;
    for (int k = 0; k < nparts; ++k) a += parts[k];
    st->delta = a;
    st->iters += 1;
    st->cur ^= 1;
    if (!isfinite(a)) st->done = 3;
    else if (a * d / (1.0 - d) < tol) st->done = 1;
    else if (st->iters >= max_iter) st->done = 2;
}

// device address of the static array, looked up once per device (host code cannot use
// the array's name as a device address)
std::mutex g_na_mutex;
unsigned char *g_na_ptr[64] = {nullptr};

di_status na_scratch(unsigned char **out) {
    int dev = 0;
    DI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(DI_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return DI_OK;
}

// device memory of the current GPU, or managed memory; another GPU's memory is rejected
// because the kernels would reach it only through peer access that may not be enabled
bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace diter

using namespace diter;

extern "C" di_status di_power_noalloc(int32_t n, const int32_t *in_ptr, const int32_t *in_src, int64_t nnz,
                                      const int32_t *row_ptr, double d, double tol, int32_t max_iter, double *X_out,
                                      di_stats *stats, void *stream) {
    if (n < 1 || n > kNaMaxN)
        return set_error(DI_EINVAL, "di_power_noalloc: n must be in [1, 65536] (the size of its static work area)");
    if (nnz < 0 || nnz >= INT32_MAX) return set_error(DI_EINVAL, "di_power_noalloc: nnz must be in [0, 2^31-1)");
    if (!in_ptr || !row_ptr || !X_out || (nnz > 0 && !in_src))
        return set_error(DI_EINVAL, "di_power_noalloc: NULL pointer");
    if (!(d > 0.0 && d < 1.0)) return set_error(DI_EINVAL, "di_power_noalloc: d must satisfy 0 < d < 1");
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(DI_EINVAL, "di_power_noalloc: tol must be finite and > 0");
    if (!on_device(in_ptr) || (nnz > 0 && !on_device(in_src)) || !on_device(row_ptr) || !on_device(X_out))
        return set_error(DI_EINVAL, "di_power_noalloc: every array must be device memory of the current GPU");
    if (max_iter <= 0) max_iter = 100000;
    unsigned char *base = nullptr;
    di_status r = na_scratch(&base);
    if (r != DI_OK) return r;
    NaState *st = reinterpret_cast<NaState *>(base);
    double *parts = reinterpret_cast<double *>(base + kNaOffParts);
    double *Z0 = reinterpret_cast<double *>(base + kNaOffZ0);
    double *Z1 = reinterpret_cast<double *>(base + kNaOffZ1);
    cudaStream_t s = (cudaStream_t)stream;
    const int nparts = std::max(1, std::min(kNaMaxParts, (n + kNaThreads - 1) / kNaThreads));
    const auto t0 = std::chrono::steady_clock::now();
    NaState h{};
    DI_CUDA(cudaMemsetAsync(&st->flags, 0, sizeof(int), s));  // the array keeps the last call's contents
    k_na_check_ptrs<<<nparts, kNaThreads, 0, s>>>(n, nnz, in_ptr, row_ptr, st);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(&h, st, sizeof(NaState), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if (h.flags & 1) return set_error(DI_EINVAL, "di_power_noalloc: in_ptr is not a valid CSR pointer array for nnz");
    if (h.flags & 2) return set_error(DI_EINVAL, "di_power_noalloc: row_ptr is not a valid CSR pointer array for nnz");
    if (nnz > 0) {
        k_na_check_src<<<nparts, kNaThreads, 0, s>>>(n, nnz, in_src, st);
        DI_CUDA(cudaGetLastError());
        DI_CUDA(cudaMemcpyAsync(&h, st, sizeof(NaState), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        if (h.flags & 4) return set_error(DI_EINVAL, "di_power_noalloc: in_src has an id outside [0, n)");
    }
    k_na_init<<<nparts, kNaThreads, 0, s>>>(n, X_out, Z0, Z1, st);
    DI_CUDA(cudaGetLastError());
    long long launches = nnz > 0 ? 3 : 2;  // the checks and the initialization
    for (int done_iters = 0; done_iters < max_iter; done_iters += kNaBatch) {
        for (int k = 0; k < kNaBatch; ++k) {
            k_na_pull<<<nparts, kNaThreads, 0, s>>>(n, in_ptr, in_src, row_ptr, d, X_out, Z0, Z1, parts, st);
            k_na_finalize<<<1, 32, 0, s>>>(nparts, parts, d, tol, max_iter, st);
            launches += 2;
        }
        DI_CUDA(cudaGetLastError());
        DI_CUDA(cudaMemcpyAsync(&h, st, sizeof(NaState), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        if (h.done) break;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) {
        stats->bound = h.delta * d / (1.0 - d);
        stats->l1_F = h.delta;
        stats->R = h.delta;
        stats->edges_pushed = (int64_t)h.iters * nnz;
        stats->sources_pushed = (int64_t)h.iters * n;
        stats->sweeps = h.iters;
        stats->converged = h.done == 1 ? 1 : 0;
        stats->seconds = secs;
        stats->kernel_launches = launches;
    }
    if (h.done == 3) return set_error(DI_EKERNEL, "di_power_noalloc: iteration became non-finite");
    if (h.done != 1) return set_error(DI_ENOTCONVERGED, "di_power_noalloc: max_iter reached before the stop rule");
    return DI_OK;
}
